"""Pins of the oracle's micromagnetic energy (oracle/micromag.py) against closed
forms: the exchange energy and field of a spin spiral, the demag energy of a
uniformly magnetized cube (mu0 Ms^2 V / 6 from the self term N = 1/3), the
Stoner-Wohlfarth energy of a single cell, and the effective field as minus the
energy gradient (central differences)."""
import numpy as np
import pytest

from oracle import micromag as omm
from oracle import newell as onw

MU0 = 4e-7 * np.pi


def test_exchange_of_a_spin_spiral():
    """m = (cos k x, sin k x, 0): every x-neighbour pair has |dm|^2 = 2 - 2 cos(k dx),
    y-neighbours none; the discrete Laplacian of the spiral is -(2 - 2 cos k dx)/dx^2 m
    in the interior."""
    nx, ny, dx, dy, dz, A, Js = 17, 5, 2e-9, 3e-9, 1e-9, 1.3e-11, 1.2
    k = 2 * np.pi / (11 * dx)
    x = np.arange(nx) * dx
    m = np.zeros((3, ny, nx))
    m[0] = np.cos(k * x)[None, :]
    m[1] = np.sin(k * x)[None, :]
    mask = np.ones((ny, nx), bool)
    V = dx * dy * dz
    want = A * V * (nx - 1) * ny * (2 - 2 * np.cos(k * dx)) / dx ** 2
    assert omm.exchange_energy(m, mask, dx, dy, A, dz) == pytest.approx(want, rel=1e-12)
    zero = np.zeros((3, ny, nx))
    b = omm.effective_field(m, mask, dx, dy, Js, A, 0.0, [0, 0, 0], zero, zero)
    lam = (2 * A * MU0 / Js) * (2 * np.cos(k * dx) - 2) / dx ** 2
    assert np.allclose(b[:, :, 1:-1], lam * m[:, :, 1:-1], rtol=1e-10, atol=1e-12 * abs(lam))
    # a boundary cell has one neighbour: (m_1 - m_0) / dx^2 only
    edge = (2 * A * MU0 / Js) * (m[:, :, 1] - m[:, :, 0]) / dx ** 2
    assert np.allclose(b[:, :, 0], edge, rtol=1e-12, atol=1e-12 * abs(lam))


def test_uniform_cube_demag_energy_is_mu0_ms2_v_over_6():
    """A single cubic cell: b_self = -Js N m with N = 1/3 (the oracle tensor's self
    term), E_d = mu0 Ms^2 V / 6 for any direction of m."""
    d = 2e-9
    N = onw.tensor(0.0, 0.0, 0.0, (2.0, 2.0, 2.0), (2.0, 2.0, 2.0))
    Js = 1.75
    Ms = Js / MU0
    for mv in ([0, 0, 1], [1, 0, 0], [0.6, 0.0, 0.8]):
        m = np.array(mv, float).reshape(3, 1, 1)
        Nm = np.array([[N[0], N[3], N[4]], [N[3], N[1], N[5]], [N[4], N[5], N[2]]]) @ m[:, 0, 0]
        b_self = (-Js * Nm).reshape(3, 1, 1)
        E = omm.energy(m, np.ones((1, 1), bool), d, d, d, Js, 0.0, 0.0, [0, 0, 0], b_self, np.zeros((3, 1, 1)))
        assert E == pytest.approx(MU0 * Ms ** 2 * d ** 3 / 6, rel=1e-12)


def test_single_cell_stoner_wohlfarth_energy():
    """One cell, m at angle theta from z in the x-z plane, field b along z, demag
    tensor diag(Nxx, Nxx, Nzz): E / V = -Ku cos^2 + mu0 Ms^2 (Nzz cos^2 + Nxx sin^2) / 2
    - Ms b cos."""
    dx, dz = 2e-9, 0.8e-9
    N = onw.tensor(0.0, 0.0, 0.0, (2.0, 2.0, 0.8), (2.0, 2.0, 0.8))
    Js, Ku, b = 1.75, 2.09e6, -0.3
    Ms = Js / MU0
    V = dx * dx * dz
    for th in np.linspace(0, np.pi, 7):
        m = np.array([np.sin(th), 0.0, np.cos(th)]).reshape(3, 1, 1)
        b_self = (-Js * np.array([N[0] * m[0, 0, 0], 0.0, N[2] * m[2, 0, 0]])).reshape(3, 1, 1)
        E = omm.energy(m, np.ones((1, 1), bool), dx, dx, dz, Js, 0.0, Ku, [0, 0, b], b_self, np.zeros((3, 1, 1)))
        want = V * (-Ku * np.cos(th) ** 2 + 0.5 * MU0 * Ms ** 2 * (N[2] * np.cos(th) ** 2 + N[0] * np.sin(th) ** 2)
                    - Ms * b * np.cos(th))
        assert E == pytest.approx(want, rel=1e-12, abs=1e-12 * abs(want) + 1e-40)


def test_effective_field_is_minus_the_energy_gradient():
    """b_eff = -(mu0 / (Js V)) dE/dm, by central differences of the energy, with
    every term on (a masked layer, random m, random bias and self fields taken
    from a symmetric operator so that the 1/2 of the self term applies)."""
    rng = np.random.default_rng(3)
    ny, nx = 6, 7
    dx, dy, dz, Js, A, Ku = 1.5e-9, 2e-9, 1e-9, 1.4, 1.1e-11, 3e5
    mask = np.ones((ny, nx), bool)
    mask[0, :2] = False
    mask[4, 5] = False
    m = rng.standard_normal((3, ny, nx))
    m /= np.linalg.norm(m, axis=0)
    m *= mask
    n = 3 * ny * nx
    S = rng.standard_normal((n, n)) * 0.05
    S = S + S.T  # a symmetric self-field operator b_self = S m
    b_bias = rng.standard_normal((3, ny, nx)) * 0.1
    b_ext = [0.02, -0.01, 0.3]
    V = dx * dy * dz

    def E(mm):
        bs = (S @ mm.ravel()).reshape(3, ny, nx)
        return omm.energy(mm, mask, dx, dy, dz, Js, A, Ku, b_ext, bs, b_bias)

    bs = (S @ m.ravel()).reshape(3, ny, nx)
    b = omm.effective_field(m, mask, dx, dy, Js, A, Ku, b_ext, bs, b_bias)
    h = 1e-6
    for (c, y, x) in [(0, 2, 3), (2, 1, 1), (1, 5, 6), (2, 0, 6), (0, 3, 0)]:
        mp, mm_ = m.copy(), m.copy()
        mp[c, y, x] += h
        mm_[c, y, x] -= h
        grad = (E(mp) - E(mm_)) / (2 * h)
        assert -MU0 / (Js * V) * grad == pytest.approx(b[c, y, x], rel=1e-6, abs=1e-9)
