"""FP64 CPU oracle for the NS-PNP fractional step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code,
constant tables or helpers with the CUDA library; the two sides meet only in
the tests, on the same seeded inputs.

Parity status per function (pins live in ``tests/test_oracle_*.py``):
all functions of ``pnp_oracle`` are pinned; see the module docstring there.
"""
