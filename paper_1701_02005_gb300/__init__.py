"""GB300-native NS-PNP fractional step (arXiv:1701.02005).

The compute path is libpnp (CUDA, sm_103a) behind the C ABI of include/pnp.h;
``binding`` mirrors that ABI with ctypes and ``solver.Solver`` wraps one
context with torch-owned device memory and stream.
"""
__all__ = ["binding", "solver", "build"]
