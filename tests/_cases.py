"""Shared helpers of the GPU parity tests: oracle fields on seeded inputs.

Only oracle/ computes expected values here; the CUDA path is never consulted.
"""
import functools

import numpy as np

from oracle import demag as odm
from oracle import newell as onw


@functools.lru_cache(maxsize=8)
def quad_kernels(nx, ny, dx, dy, thickness):
    """Full-offset layer kernels from the exact _Float128 tensor (the definition)."""
    return onw.layer_kernels(nx, ny, dx, dy, list(thickness), mode=onw.EXACT_Q, full=True)


@functools.lru_cache(maxsize=8)
def reading_kernels(nx, ny, dx, dy, thickness):
    """Full-offset layer kernels from the reading (double near, quadrature far),
    expanded from the quadrant by the tensor's parity in X and Y."""
    Kq = onw.layer_kernels(nx, ny, dx, dy, list(thickness), mode=onw.READING_D, full=False)
    return odm.expand_quadrant(Kq)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
