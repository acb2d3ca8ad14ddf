"""ctypes wrapper of the oracle's generalized-Newell library (test infrastructure only).

Every function here follows Sec. 2 of the paper (Eqs. Nxx, F, F_2, Nxy, G,
G2_as_g and App. A/B); the C source states each step.  Component order
everywhere: (xx, yy, zz, xy, xz, yz).
"""
import ctypes
import numpy as np

from . import build as _build

EXACT_Q = 0       # exact formula in _Float128, 64-term form (the definition)
EXACT_Q_FULL = 1  # exact formula in _Float128, 256 (N_xx) / 128 (N_xy) terms
EXACT_D = 2       # exact formula in double
FARFIELD_D = 3    # Gauss-Legendre quadrature of the volume integral, double
READING_D = 4     # exact double for near cells, composite quadrature beyond one cell gap

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_tensor.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    dp, dp, ctypes.c_int, dp, dp]
        L.oracle_tensor.restype = None
        L.oracle_newell_fg_q.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, dp, dp]
        L.oracle_newell_fg_q.restype = None
        L.oracle_newell_fg_d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double]
        L.oracle_newell_fg_d.restype = ctypes.c_double
        L.oracle_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
        L.oracle_gauss_legendre.restype = None
        L.oracle_layer_kernels.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, dp, ctypes.c_int, dp]
        L.oracle_layer_kernels.restype = None
        L.oracle_pair_kernel.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp]
        L.oracle_pair_kernel.restype = None
        L.oracle_tensor_dt.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, dp]
        L.oracle_tensor_dt.restype = None
        L.oracle_layer_dkernels.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, dp]
        L.oracle_layer_dkernels.restype = None
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def tensor(X, Y, Z, target, source, mode=EXACT_Q, nquad=4, with_lo=False):
    """Generalized demag tensor N(target <- source) at offset (X, Y, Z).

    (X, Y, Z) = target corner - source corner; target, source = (edge_x,
    edge_y, edge_z).  Normalised by the target volume (Sec. 2).  Returns
    float64[6] = (xx, yy, zz, xy, xz, yz); with_lo also returns the _Float128
    remainder (q modes) so that hi + lo carries ~32 digits.
    """
    t = np.ascontiguousarray(target, dtype=np.float64)
    s = np.ascontiguousarray(source, dtype=np.float64)
    out = np.zeros(6)
    lo = np.zeros(6)
    lib().oracle_tensor(int(mode), float(X), float(Y), float(Z), _dp(t), _dp(s), int(nquad),
                        _dp(out), _dp(lo))
    return (out, lo) if with_lo else out


def newell_f(x, y, z, quad=True):
    """Newell f (Sec. 2.1).  quad=True returns (hi, lo) of the _Float128 value."""
    if quad:
        hi, lo = ctypes.c_double(), ctypes.c_double()
        lib().oracle_newell_fg_q(0, x, y, z, ctypes.byref(hi), ctypes.byref(lo))
        return hi.value, lo.value
    return lib().oracle_newell_fg_d(0, x, y, z)


def newell_g(x, y, z, quad=True):
    """Newell g (Sec. 2.2).  quad=True returns (hi, lo) of the _Float128 value."""
    if quad:
        hi, lo = ctypes.c_double(), ctypes.c_double()
        lib().oracle_newell_fg_q(1, x, y, z, ctypes.byref(hi), ctypes.byref(lo))
        return hi.value, lo.value
    return lib().oracle_newell_fg_d(1, x, y, z)


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().oracle_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def layer_kernels(nx, ny, dx, dy, thickness, mode=READING_D, full=True):
    """All layer-pair convolution kernels of the layer stack (Sec. 3).

    Returns K with K[i, j, c, q, p] = N_c(i <- j) at in-plane offset
    (p' dx, q' dy) where p' = p - (nx - 1), q' = q - (ny - 1) if full (shape
    [L, L, 6, 2ny-1, 2nx-1]), else p' = p, q' = q (shape [L, L, 6, ny, nx]).
    Layers are stacked from z = 0 upward; layer i has thickness thickness[i].
    """
    th = np.ascontiguousarray(thickness, dtype=np.float64)
    L = th.size
    shape = (L, L, 6, 2 * ny - 1, 2 * nx - 1) if full else (L, L, 6, ny, nx)
    K = np.zeros(shape)
    lib().oracle_layer_kernels(int(mode), int(nx), int(ny), float(dx), float(dy), int(L), _dp(th),
                               1 if full else 0, _dp(K))
    return K


def tensor_dt(X, Y, Z, target, source, dtz, dsz, dZ, h=1e-9):
    """d N(target <- source) along (target z-edge, source z-edge, z-offset),
    central difference of the exact _Float128 tensor with step h."""
    t = np.ascontiguousarray(target, dtype=np.float64)
    s = np.ascontiguousarray(source, dtype=np.float64)
    out = np.zeros(6)
    lib().oracle_tensor_dt(float(X), float(Y), float(Z), _dp(t), _dp(s), float(dtz), float(dsz),
                           float(dZ), float(h), _dp(out))
    return out


def layer_dkernels(nx, ny, dx, dy, thickness, layer, h=1e-9):
    """d/d t_layer of layer_kernels(full=True) (exact tensor, _Float128 differences)."""
    th = np.ascontiguousarray(thickness, dtype=np.float64)
    L = th.size
    K = np.zeros((L, L, 6, 2 * ny - 1, 2 * nx - 1))
    lib().oracle_layer_dkernels(int(nx), int(ny), float(dx), float(dy), int(L), _dp(th), int(layer),
                                float(h), _dp(K))
    return K


def pair_kernel(nx, ny, dx, dy, thickness, i, j, mode=READING_D):
    """Kernel of one layer pair (target i, source j) at every in-plane offset:
    [6, 2ny-1, 2nx-1], offset index + n - 1 (as layer_kernels(full=True)[i, j])."""
    th = np.ascontiguousarray(thickness, dtype=np.float64)
    K = np.zeros((6, 2 * ny - 1, 2 * nx - 1))
    lib().oracle_pair_kernel(int(mode), int(nx), int(ny), float(dx), float(dy), int(th.size), _dp(th),
                             int(i), int(j), _dp(K))
    return K
