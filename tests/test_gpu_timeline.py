"""pnp_timeline: one traced step in the step's concurrent schedule, launched
eagerly or as one CUDA graph with the timing events as graph nodes.

The trace lists every launch site once per substage on the stream that ran
it (the ion CN solve and the potential pipeline on the auxiliary stream, the
rest on the context's stream), its event times never decrease along a stream,
and the traced step advances the state exactly as pnp_step does.
"""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o

pytestmark = pytest.mark.gpu


def _mixed(g, prm):
    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, y_faces=g.yf, precision=B.PNP_MIXED)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta)
    return s


@pytest.mark.parametrize("in_graph", [False, True])
def test_timeline_covers_every_site_and_matches_a_step(in_graph):
    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import timeline

    g = o.Grid(64, 33, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=400.0, lam=0.05, V=2.0)
    a, b = _mixed(g, prm), _mixed(g, prm)
    for s in (a, b):
        s.init_state(B.PNP_IC_PB, 11, 1e-2)
        s.step(2, 0.01)
    a.step(1, 0.01)
    tr = timeline(b, 0.01, in_graph=in_graph)
    assert [e[0] for e in tr].count("start") == 3
    per = len(tr) // 3
    assert len(tr) == 3 * per == 45
    for l in range(3):
        sub = tr[l * per:(l + 1) * per]
        assert sub[0][0] == "start" and sub[1][0] == "rhs" and sub[1][1] == "main"
        names = [e[0] for e in sub[1:]]
        assert sorted(names) == sorted(list(B.PROFILE_SITES) + ["cn_thomas"])
        for name, stream, _ in sub[2:]:
            if name.startswith("e_"):
                assert stream == "aux", name
            elif name != "cn_thomas":
                assert stream == "main", name
        assert sorted(st for n, st, _ in sub if n == "cn_thomas") == ["aux", "main"]
    for stream in ("main", "aux"):
        t = [e[2] for e in tr if e[1] == stream]
        assert all(t1 >= t0 for t0, t1 in zip(t, t[1:])), stream
    assert tr[-1][2] > 0.0
    for name in ("u", "v", "w", "cp", "cm", "Phi"):
        assert np.array_equal(a.get(name), b.get(name)), name
    a.close()
    b.close()
