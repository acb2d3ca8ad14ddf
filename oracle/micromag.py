"""Oracle micromagnetic energy of one magnetic layer of the stack (test
infrastructure only; the CUDA library never imports it).

Sec. 4 of the paper relaxes the free layer of the MRAM stack with a
limited-memory BFGS energy minimisation for every applied field of an
easy-axis hysteresis loop, with exchange, uniaxial anisotropy (easy axis z),
the applied (Zeeman) field and the demagnetization field of the whole stack
(the pinned layers' stray field and the layer's own field).  These are the
plain textbook definitions of those terms on the cell grid, in SI units:

* exchange      E_ex = A V sum_i sum_{j nb i} |m_j - m_i|^2 / (2 d_ij^2)
                (nearest in-plane neighbours inside the layer's mask; a
                neighbour outside the mask contributes nothing: free surface)
* anisotropy    E_an = -K_u V sum_i (m_i . e_z)^2
* Zeeman        E_z  = -(J_s / mu0) V sum_i m_i . b_ext
* demag         E_d  = -(J_s / mu0) V sum_i m_i . (b_self,i / 2 + b_bias,i)

with V the cell volume, J_s = mu0 M_s, fields b in tesla (mu0 H), b_self the
field of the layer's own magnetization and b_bias that of the other (fixed)
layers.  The effective field is b_eff,i = -(mu0 / (J_s V)) dE/dm_i:

    b_eff = (2 A mu0 / J_s) sum_j (m_j - m_i) / d_ij^2 + (2 K_u mu0 / J_s) m_z e_z
            + b_ext + b_self + b_bias

(the demag self-term's factor 1/2 disappears because the layer's own demag
operator is symmetric: target and source cells have one thickness).
"""
import numpy as np

MU0 = 4e-7 * np.pi


def exchange_energy(m, mask, dx, dy, A, dz):
    """E_ex of a layer m [3, ny, nx] (unit vectors in the mask), cell dx x dy x dz (m)."""
    V = dx * dy * dz
    E = 0.0
    for axis, d in ((2, dx), (1, dy)):
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[axis] = slice(1, None)
        b[axis] = slice(None, -1)
        both = mask[tuple(a[1:])] & mask[tuple(b[1:])]
        diff = m[tuple(a)] - m[tuple(b)]
        # every neighbouring pair once: sum over i of sum over nb j / 2 counts each pair once
        E += A * V * np.sum(np.sum(diff ** 2, axis=0)[both]) / d ** 2
    return float(E)


def energy(m, mask, dx, dy, dz, Js, A, Ku, b_ext, b_self, b_bias):
    """Total energy (J) of the layer m [3, ny, nx]; fields [3, ny, nx] or [3] in tesla."""
    V = dx * dy * dz
    Ms = Js / MU0
    w = mask.astype(np.float64)
    b_ext = np.broadcast_to(np.asarray(b_ext, dtype=np.float64).reshape(3, *([1] * (m.ndim - 1))), m.shape)
    E_an = -Ku * V * np.sum(w * m[2] ** 2)
    E_z = -Ms * V * np.sum(w * np.sum(m * b_ext, axis=0))
    E_d = -Ms * V * np.sum(w * np.sum(m * (0.5 * b_self + b_bias), axis=0))
    return exchange_energy(m, mask, dx, dy, A, dz) + float(E_an) + float(E_z) + float(E_d)


def effective_field(m, mask, dx, dy, Js, A, Ku, b_ext, b_self, b_bias):
    """b_eff (tesla) [3, ny, nx], zero outside the mask."""
    lap = np.zeros_like(m)
    for axis, d in ((2, dx), (1, dy)):
        for shift in (1, -1):
            nb = np.roll(m, shift, axis=axis)
            nmask = np.roll(mask, shift, axis=axis - 1)
            # np.roll wraps around: the wrapped row or column is not a neighbour
            edge = [slice(None)] * 2
            edge[axis - 1] = slice(0, 1) if shift == 1 else slice(-1, None)
            nmask = nmask.copy()
            nmask[tuple(edge)] = False
            lap += np.where(nmask & mask, nb - m, 0.0) / d ** 2
    b_ext = np.asarray(b_ext, dtype=np.float64).reshape(3, 1, 1)
    b = (2 * A * MU0 / Js) * lap + b_ext + b_self + b_bias
    b[2] += (2 * Ku * MU0 / Js) * m[2]
    return np.where(mask, b, 0.0)
