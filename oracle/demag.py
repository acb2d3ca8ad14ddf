"""Oracle demagnetization field of a non-equidistant layer stack (test infrastructure only).

Plain float64 numpy restatements of Sec. 3 of the paper:

* ``direct_sum``   Eq. Hi_discrete: H_i = -Ms sum_j N_{i-j} m_j over every cell
                   pair, including i = j, by explicit loops over the in-plane
                   offsets.
* ``hybrid``       Eq. FFT_v2: 2D FFTs over x and y, an explicit sum over the
                   layers j per frequency, inverse 2D FFT, crop and -Ms scaling.
* ``fft3d``        Eq. FFT_3D: the equidistant method (all layers of one
                   thickness), FFTs over x, y and z.

Arrays: magnetization m and field H are [L, 3, ny, nx] (or [B, L, 3, ny, nx]),
x fastest, component order (x, y, z).  Layer kernels K come from
``oracle.newell.layer_kernels`` with the component order
(xx, yy, zz, xy, xz, yz) and K[i, j] = N(i <- j) (target layer i, source j).
"""
import numpy as np

# 3x3 block position -> packed component index (the tensor is symmetric, Sec. 2)
_COMP = ((0, 3, 4), (3, 1, 5), (4, 5, 2))


def expand_quadrant(Kq):
    """Full kernels [L, L, 6, 2ny-1, 2nx-1] from the quadrant [L, L, 6, ny, nx].

    Uses the parity of the generalized tensor in the in-plane offsets when the
    in-plane cell sizes of source and target agree: f is even and g odd in x
    and y (Sec. 2.1, 2.2), so N_xx, N_yy, N_zz are even in X and Y, N_xy is odd
    in both, N_xz odd in X / even in Y, N_yz even in X / odd in Y.
    """
    L1, L2, C, ny, nx = Kq.shape
    sx = np.array([1, 1, 1, -1, -1, 1], dtype=np.float64)  # sign under X -> -X
    sy = np.array([1, 1, 1, -1, 1, -1], dtype=np.float64)  # sign under Y -> -Y
    qs = np.arange(-(ny - 1), ny)
    ps = np.arange(-(nx - 1), nx)
    K = Kq[:, :, :, np.abs(qs)[:, None], np.abs(ps)[None, :]]
    sgn_x = np.where(ps[None, :] < 0, sx[:, None], 1.0)  # [6, 2nx-1]
    sgn_y = np.where(qs[None, :] < 0, sy[:, None], 1.0)  # [6, 2ny-1]
    return K * (sgn_y[:, :, None] * sgn_x[:, None, :])


def direct_sum(K, m, Ms):
    """Eq. Hi_discrete by brute force: H_i = -Ms sum_j N(i <- j) m_j.

    K: full layer kernels [L, L, 6, 2ny-1, 2nx-1] (offset index + n - 1).
    m: [L, 3, ny, nx] or [B, L, 3, ny, nx].
    """
    m = np.asarray(m, dtype=np.float64)
    batched = m.ndim == 5
    mb = m if batched else m[None]
    B, L, _, ny, nx = mb.shape
    H = np.zeros_like(mb)
    for q in range(-(ny - 1), ny):
        ys_t = slice(max(0, q), min(ny, ny + q))
        ys_s = slice(max(0, -q), min(ny, ny - q))
        for p in range(-(nx - 1), nx):
            xs_t = slice(max(0, p), min(nx, nx + p))
            xs_s = slice(max(0, -p), min(nx, nx - p))
            for i in range(L):
                for j in range(L):
                    n = K[i, j, :, q + ny - 1, p + nx - 1]
                    src = mb[:, j, :, ys_s, xs_s]
                    for a in range(3):
                        acc = 0.0
                        for b in range(3):
                            acc = acc + n[_COMP[a][b]] * src[:, b]
                        H[:, i, a, ys_t, xs_t] += acc
    H *= -Ms
    return H if batched else H[0]


def padded_kernel_spectra(K):
    """2D FFTs of the layer kernels zero-padded to the 2nx x 2ny circulant grid.

    Offset p in (-nx, nx) goes to index p mod 2nx; index nx (no offset within
    the grid reaches it) stays zero.  Returns complex [L, L, 6, 2ny, 2nx].
    """
    L1, L2, C, qh, pw = K.shape
    ny, nx = (qh + 1) // 2, (pw + 1) // 2
    Kp = np.zeros((L1, L2, C, 2 * ny, 2 * nx))
    qs = np.arange(-(ny - 1), ny) % (2 * ny)
    ps = np.arange(-(nx - 1), nx) % (2 * nx)
    Kp[:, :, :, qs[:, None], ps[None, :]] = K
    return np.fft.fft2(Kp, axes=(-2, -1))


def hybrid(K, m, Ms, Khat=None):
    """Eq. FFT_v2: FFT in x and y, explicit convolution over the layers.

    H_i = -Ms F^-1 [ sum_j F(N_ij) F(m_j) ], cropped to the grid.
    K as in direct_sum (ignored when Khat, from padded_kernel_spectra, is given).
    """
    m = np.asarray(m, dtype=np.float64)
    batched = m.ndim == 5
    mb = m if batched else m[None]
    B, L, _, ny, nx = mb.shape
    if Khat is None:
        Khat = padded_kernel_spectra(K)
    mp = np.zeros((B, L, 3, 2 * ny, 2 * nx))
    mp[..., :ny, :nx] = mb
    mhat = np.fft.fft2(mp, axes=(-2, -1))
    Hhat = np.zeros_like(mhat)
    for i in range(L):
        for j in range(L):
            for a in range(3):
                for b in range(3):
                    Hhat[:, i, a] += Khat[i, j, _COMP[a][b]] * mhat[:, j, b]
    H = np.fft.ifft2(Hhat, axes=(-2, -1)).real[..., :ny, :nx] * (-Ms)
    return H if batched else H[0]


def fft3d(Kz, m, Ms):
    """Eq. FFT_3D for the equidistant stack (all layers one thickness).

    Kz: kernels by layer offset r = i - j in (-L, L), shape [2L-1, 6, 2ny-1, 2nx-1]
    with Kz[r + L - 1] = N(target layer i <- source layer i - r).
    """
    m = np.asarray(m, dtype=np.float64)
    batched = m.ndim == 5
    mb = m if batched else m[None]
    B, L, _, ny, nx = mb.shape
    Kp = np.zeros((6, 2 * L, 2 * ny, 2 * nx))
    rs = np.arange(-(L - 1), L) % (2 * L)
    qs = np.arange(-(ny - 1), ny) % (2 * ny)
    ps = np.arange(-(nx - 1), nx) % (2 * nx)
    Kp[:, rs[:, None, None], qs[None, :, None], ps[None, None, :]] = np.moveaxis(Kz, 1, 0)
    Khat = np.fft.fftn(Kp, axes=(-3, -2, -1))
    mp = np.zeros((B, 3, 2 * L, 2 * ny, 2 * nx))
    mp[:, :, :L, :ny, :nx] = np.moveaxis(mb, 1, 2)
    mhat = np.fft.fftn(mp, axes=(-3, -2, -1))
    Hhat = np.zeros_like(mhat)
    for a in range(3):
        for b in range(3):
            Hhat[:, a] += Khat[_COMP[a][b]] * mhat[:, b]
    H = np.fft.ifftn(Hhat, axes=(-3, -2, -1)).real[:, :, :L, :ny, :nx] * (-Ms)
    H = np.moveaxis(H, 2, 1)
    return H if batched else H[0]


def hybrid_targets(pair_kernel, m, Ms, targets):
    """Eq. FFT_v2 for selected target layers only, one layer pair at a time
    (bounded memory for large stacks): H_i for i in targets.

    pair_kernel(i, j) -> [6, 2ny-1, 2nx-1] kernel of the pair; m: [L, 3, ny, nx].
    Returns {i: H_i [3, ny, nx]}.
    """
    m = np.asarray(m, dtype=np.float64)
    L, _, ny, nx = m.shape
    mp = np.zeros((L, 3, 2 * ny, 2 * nx))
    mp[..., :ny, :nx] = m
    mhat = np.fft.fft2(mp, axes=(-2, -1))
    qs = np.arange(-(ny - 1), ny) % (2 * ny)
    ps = np.arange(-(nx - 1), nx) % (2 * nx)
    out = {}
    for i in targets:
        Hhat = np.zeros((3, 2 * ny, 2 * nx), dtype=complex)
        for j in range(L):
            Kp = np.zeros((6, 2 * ny, 2 * nx))
            Kp[:, qs[:, None], ps[None, :]] = pair_kernel(i, j)
            Khat = np.fft.fft2(Kp, axes=(-2, -1))
            for a in range(3):
                for b in range(3):
                    Hhat[a] += Khat[_COMP[a][b]] * mhat[j, b]
        out[i] = np.fft.ifft2(Hhat, axes=(-2, -1)).real[..., :ny, :nx] * (-Ms)
    return out
