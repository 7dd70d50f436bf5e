"""Host logic of bench.py (no GPU): the per-cell algorithmic byte model behind
the roofline figures and the ensemble recipe."""
import bench


def test_mixed_byte_model():
    half = (bench.WL["nx"] // 2 + 1) / bench.WL["nx"]
    c = lambda s, cfg=None: bench.site_cost(s, "mixed", cfg)["bytes"]
    # stencil: 28 B of inputs + 20 B of right-hand sides, plus the previous H
    # (20 B) in two substages of three and the new H (20 B) in two of three
    assert abs(c("rhs") - (28 + 20 + 20 * 2 / 3 + 20 * 2 / 3)) < 1e-12
    # CN: the back substitution after the stencil's fused forward elimination (the
    # default) and the shared-memory tiles (launch code 32) move 76 B per cell; the
    # unfused line kernels write and re-read the forward values (116 B)
    unfused = lambda cfg: bench.site_cost("cn_thomas", "mixed", cfg, False)["bytes"]
    assert c("cn_thomas") == 76 and c("cn_thomas", [64, 32, 32, 16]) == 76
    assert unfused([64, 64, 32, 16]) == 116 and unfused([64, 32, 32, 16]) == 76
    # a spectral y-solve: spectrum in / out (8 + 8), df forward values out / in
    # (16 + 16) and the df factors (16) per spectral point
    assert abs(c("p_thomas") - 64 * half) < 1e-12 and abs(c("e_thomas") - 64 * half) < 1e-12
    sites = ("rhs", "cn_thomas", "p_fftx", "p_fftz", "p_thomas", "p_ifftz", "p_ifftx", "project",
             "e_fftx", "e_fftz", "e_thomas", "e_ifftz", "e_ifftx")
    total = sum(c(s) for s in sites)
    assert 325 < total < 332   # ~328 B per cell and substage with the fused CN forward elimination
    # the measured stencil traffic is quoted for the default stencil kernel
    nt = bench.NCU_TRAFFIC[("mixed", "rhs")]
    assert nt["shape"] == (0, 64) and nt["cells"] == bench.cells()
    assert 0.9 < nt["bytes"] / (c("rhs") * bench.cells()) < 1.0


def test_ensemble_recipe():
    cases = bench.ensemble_cases()
    assert len(cases) == 48
    assert sum(bench.cells(c) for c in cases) == 44_040_192
    assert {(c["nx"], c["ny"], c["nz"]) for c in cases} == {(64, 65, 64), (128, 97, 128)}


def test_reference_arm_prints_one_contract_line():
    # bench.py --impl reference times the oracle on the host: one JSON line with
    # the contract's keys (a tiny grid override keeps it to a few seconds)
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--grid", "16,17,16",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
