"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Random numbers only: nothing here computes any part of the NS-PNP method.
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def field(seed, shape, scale=1.0, offset=0.0):
    return offset + scale * rng(seed).standard_normal(shape)


def positive_field(seed, shape, lo=0.5, hi=1.5):
    return rng(seed).uniform(lo, hi, size=shape)


def wall_zero_faces(seed, shape, scale=1.0):
    """Random face field with zero first and last planes (v on the walls)."""
    a = field(seed, shape, scale)
    a[0] = 0.0
    a[-1] = 0.0
    return a


def diag_dominant_rows(seed, n, complex_rhs=False, nrhs=7):
    r = rng(seed)
    a = r.uniform(-1, 1, n)
    c = r.uniform(-1, 1, n)
    a[0] = 0.0
    c[-1] = 0.0
    b = (np.abs(a) + np.abs(c) + r.uniform(0.1, 2.0, n)) * r.choice([-1.0, 1.0], n)
    d = r.standard_normal((n, nrhs))
    if complex_rhs:
        d = d + 1j * r.standard_normal((n, nrhs))
    return a, b, c, d
