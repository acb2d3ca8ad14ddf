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


@functools.lru_cache(maxsize=4)
def offset_kernels(nx, ny, dx, dy, dz, nz):
    """Kernels of the z-offsets r in (-nz, nz) of an equidistant stack (Eq. FFT_3D),
    [2nz-1, 6, 2ny-1, 2nx-1] with index r + nz - 1: N(i <- i - r), from the
    reading's layer kernels (target r, source 0 for r >= 0; target 0, source -r
    below)."""
    K = reading_kernels(nx, ny, dx, dy, (float(dz),) * nz)
    return np.stack([K[r, 0] if r >= 0 else K[0, -r] for r in range(-(nz - 1), nz)])
