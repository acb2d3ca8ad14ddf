"""Pins of the oracle's generalized Newell tensor against what the mathematics fixes.

None of these re-types the oracle's formulas: each checks a property that a
dropped term, a wrong sign, a wrong shift or a transposed argument would break
(defining derivatives, a published closed form, the dipole limit, additivity,
reciprocity, symmetry under axis permutation).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import newell as nw

COMPS = ("xx", "yy", "zz", "xy", "xz", "yz")
PAIRS = [((2.0, 2.0, 1.0), (2.0, 2.0, 0.5)),
         ((2.0, 2.0, 0.5), (2.0, 2.0, 2.0)),
         ((1.5, 2.5, 0.7), (1.2, 0.8, 4.0)),   # fully unequal cuboids
         ((2.0, 2.0, 5.0), (2.0, 2.0, 1.0))]
OFFSETS = [(0.0, 0.0, 0.0), (2.0, 0.0, 0.0), (2.0, -4.0, 1.0), (-6.0, 2.0, -3.5),
           (0.3, 1.1, -0.4), (10.0, 7.0, 2.5)]


def _mp(hilo):
    import mpmath
    return mpmath.mpf(hilo[0]) + mpmath.mpf(hilo[1])


@pytest.mark.parametrize("pt", [(0.7, 1.3, 0.9), (2.0, 0.4, 1.7), (-1.1, 0.8, 2.2)])
def test_f_g_defining_derivatives(pt):
    """d^2/dy^2 d^2/dz^2 f = 1/R (Eq. F2) and d/dx d/dy d^2/dz^2 g = 1/R (Eq. G2),
    by central differences of the _Float128 f and g in 40-digit arithmetic."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    x, y, z = pt
    h = 1e-4
    R = mpmath.sqrt(mpmath.mpf(x) ** 2 + mpmath.mpf(y) ** 2 + mpmath.mpf(z) ** 2)
    c2 = {-1: 1, 0: -2, 1: 1}
    # f: second difference in y and in z
    acc = mpmath.mpf(0)
    for a, ca in c2.items():
        for b, cb in c2.items():
            acc += ca * cb * _mp(nw.newell_f(x, y + a * h, z + b * h))
    d_f = acc / mpmath.mpf(h) ** 4
    assert abs(d_f - 1 / R) / (1 / R) < 1e-6
    # g: first differences in x and y, second difference in z
    c1 = {-1: -0.5, 1: 0.5}
    acc = mpmath.mpf(0)
    for a, ca in c1.items():
        for b, cb in c1.items():
            for c, cc in c2.items():
                acc += ca * cb * cc * _mp(nw.newell_g(x + a * h, y + b * h, z + c * h))
    d_g = acc / mpmath.mpf(h) ** 4
    assert abs(d_g - 1 / R) / (1 / R) < 1e-6


def test_f_even_g_odd():
    """f is even in every argument; g is odd in x and y and even in z."""
    for (x, y, z) in [(0.7, 1.3, 0.9), (2.0, 0.4, 1.7)]:
        f0 = nw.newell_f(x, y, z, quad=False)
        for sx, sy, sz in itertools.product((1, -1), repeat=3):
            assert nw.newell_f(sx * x, sy * y, sz * z, quad=False) == pytest.approx(f0, rel=1e-14)
            g = nw.newell_g(sx * x, sy * y, sz * z, quad=False)
            assert g == pytest.approx(sx * sy * nw.newell_g(x, y, z, quad=False), rel=1e-14)


def _aharoni_nzz(A, B, C):
    """Aharoni, J. Appl. Phys. 83, 3432 (1998): demagnetizing factor along z of a
    uniformly magnetized rectangular prism of edges A x B x C (closed form)."""
    a, b, c = A / 2, B / 2, C / 2
    r = math.sqrt(a * a + b * b + c * c)
    ab, bc, ac = math.hypot(a, b), math.hypot(b, c), math.hypot(a, c)
    s = ((b * b - c * c) / (2 * b * c) * math.log((r - a) / (r + a))
         + (a * a - c * c) / (2 * a * c) * math.log((r - b) / (r + b))
         + b / (2 * c) * math.log((ab + a) / (ab - a)) + a / (2 * c) * math.log((ab + b) / (ab - b))
         + c / (2 * a) * math.log((bc - b) / (bc + b)) + c / (2 * b) * math.log((ac - a) / (ac + a))
         + 2 * math.atan(a * b / (c * r)) + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r + c / (a * b) * (ac + bc)
         - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c))
    return s / math.pi


@pytest.mark.parametrize("edges", [(1.0, 1.0, 1.0), (2.0, 2.0, 0.5), (2.0, 3.0, 0.7),
                                   (1.0, 5.0, 2.5), (3.0, 1.0, 0.2)])
def test_self_term_closed_form(edges):
    """Self term: diagonal, trace 1, each diagonal entry equal to Aharoni's
    closed form (permuting the edges gives N_xx and N_yy); 1/3 for a cube."""
    N = nw.tensor(0, 0, 0, edges, edges)
    A, B, C = edges
    assert N[2] == pytest.approx(_aharoni_nzz(A, B, C), abs=1e-13)
    assert N[0] == pytest.approx(_aharoni_nzz(B, C, A), abs=1e-13)
    assert N[1] == pytest.approx(_aharoni_nzz(C, A, B), abs=1e-13)
    assert N[:3].sum() == pytest.approx(1.0, abs=1e-14)
    assert np.all(np.abs(N[3:]) < 1e-15)
    if A == B == C:
        assert np.allclose(N[:3], 1.0 / 3.0, atol=1e-15)


def _dipole(X, Y, Z, t, s):
    c = np.array([X + (t[0] - s[0]) / 2, Y + (t[1] - s[1]) / 2, Z + (t[2] - s[2]) / 2])
    r = np.linalg.norm(c)
    D = -(np.prod(s) / (4 * np.pi)) * (3 * np.outer(c, c) - r * r * np.eye(3)) / r ** 5
    return np.array([D[0, 0], D[1, 1], D[2, 2], D[0, 1], D[0, 2], D[1, 2]])


@pytest.mark.parametrize("t,s", PAIRS)
def test_dipole_far_field(t, s):
    """Far away the tensor tends to the point-dipole field of the source,
    -(V'/4pi)(3 r r^T - r^2 I)/r^5 with r between the centres, with a relative
    error that falls as (edge / distance)^2."""
    errs = []
    for R in (40.0, 80.0, 160.0):
        X, Y, Z = 0.62 * R, 0.48 * R, 0.62 * R
        N = nw.tensor(X, Y, Z, t, s)
        D = _dipole(X, Y, Z, t, s)
        errs.append(np.abs(N - D).max() / np.abs(D).max())
    assert errs[0] < 5e-3
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0


@pytest.mark.parametrize("t,s", PAIRS)
@pytest.mark.parametrize("off", OFFSETS)
def test_axis_permutation_covariance(t, s, off):
    """Relabelling the axes of the whole problem (offsets and both cuboids)
    permutes the tensor's indices: N'_{pi(a) pi(b)} = N_{ab}.  This ties each
    permuted component (N_yy, N_zz, N_xz, N_yz) to N_xx and N_xy and checks
    N_xy = N_yx computed from the other face pairing."""
    N = nw.tensor(*off, t, s)
    M = np.array([[N[0], N[3], N[4]], [N[3], N[1], N[5]], [N[4], N[5], N[2]]])
    scale = np.abs(M).max()
    for perm in itertools.permutations(range(3)):
        offp = [off[perm[k]] for k in range(3)]
        tp = [t[perm[k]] for k in range(3)]
        sp = [s[perm[k]] for k in range(3)]
        Np = nw.tensor(*offp, tp, sp)
        Mp = np.array([[Np[0], Np[3], Np[4]], [Np[3], Np[1], Np[5]], [Np[4], Np[5], Np[2]]])
        # axis k of the permuted problem is axis perm[k] of the original
        expect = M[np.ix_(perm, perm)]
        assert np.abs(Mp - expect).max() <= 1e-14 * max(scale, 1e-3)


@pytest.mark.parametrize("t,s", PAIRS)
@pytest.mark.parametrize("off", OFFSETS)
def test_reciprocity(t, s, off):
    """|tau| N(tau <- tau')(d) = |tau'| N(tau' <- tau)(-d'): the double volume
    integral is symmetric in the two cuboids (target-volume normalisation,
    Sec. 3).  With corners, the reversed offset is -(X, Y, Z)."""
    Vt, Vs = np.prod(t), np.prod(s)
    a = Vt * nw.tensor(*off, t, s)
    b = Vs * nw.tensor(-off[0], -off[1], -off[2], s, t)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max() + 1e-16


@pytest.mark.parametrize("off", OFFSETS)
def test_source_and_target_additivity(off):
    """Splitting a cuboid in two along z splits its field (source) or its
    volume-weighted average field (target): the generalized formula must
    reproduce both identities exactly for unequal thicknesses."""
    X, Y, Z = off
    tgt = (2.0, 2.0, 0.7)
    a, b = 0.5, 1.5
    whole = nw.tensor(X, Y, Z, tgt, (2.0, 2.0, a + b))
    parts = nw.tensor(X, Y, Z, tgt, (2.0, 2.0, a)) + nw.tensor(X, Y, Z - a, tgt, (2.0, 2.0, b))
    assert np.abs(whole - parts).max() < 1e-14
    src = (2.0, 2.0, 1.3)
    whole = (a + b) * nw.tensor(X, Y, Z, (2.0, 2.0, a + b), src)
    parts = a * nw.tensor(X, Y, Z, (2.0, 2.0, a), src) + b * nw.tensor(X, Y, Z + a, (2.0, 2.0, b), src)
    assert np.abs(whole - parts).max() < 1e-14


def test_in_plane_additivity_and_cube_split():
    """A cube of edge 2 split into eight unit cubes: the self term of the big
    cube (1/3 on the diagonal) equals the volume-weighted sum of all 64 unit
    cube pair interactions divided by the big volume."""
    acc = np.zeros(6)
    corners = list(itertools.product((0.0, 1.0), repeat=3))
    for ct in corners:
        for cs in corners:
            d = [ct[k] - cs[k] for k in range(3)]
            acc += nw.tensor(*d, (1, 1, 1), (1, 1, 1))
    acc /= 8.0
    assert np.allclose(acc[:3], 1.0 / 3.0, atol=1e-14)
    assert np.all(np.abs(acc[3:]) < 1e-14)


@pytest.mark.parametrize("t,s", PAIRS[:2])
def test_64_term_form_equals_full_form(t, s):
    """The terms of Eq. F_2 constant in Y or Z, and g(X,Y,0) in Eq. G2_as_g,
    cancel in the weighted sums (end of Sec. 2.1 and 2.2)."""
    for off in OFFSETS:
        a = nw.tensor(*off, t, s, mode=nw.EXACT_Q)
        b = nw.tensor(*off, t, s, mode=nw.EXACT_Q_FULL)
        assert np.abs(a - b).max() < 1e-15


def test_gauss_legendre_rule():
    """n-point Gauss-Legendre integrates x^k exactly on [-1, 1] for k < 2n and
    matches numpy's leggauss."""
    for n in range(1, 13):
        x, w = nw.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        order = np.argsort(x)
        assert np.allclose(x[order], xr, atol=1e-14) and np.allclose(w[order], wr, atol=1e-14)
        for k in range(2 * n):
            exact = 0.0 if k % 2 else 2.0 / (k + 1)
            assert abs(np.dot(w, x ** k) - exact) < 1e-13


@pytest.mark.parametrize("t,s", PAIRS)
def test_farfield_quadrature_converges_to_exact(t, s):
    """The far-field quadrature of the volume integral converges to the exact
    _Float128 tensor as nodes are added (an independent route to the same
    definition, Eq. demag_tensor)."""
    X, Y, Z = 30.0, -22.0, 5.0
    Nq = nw.tensor(X, Y, Z, t, s)
    sc = np.abs(Nq).max()
    errs = [np.abs(nw.tensor(X, Y, Z, t, s, mode=nw.FARFIELD_D, nquad=n) - Nq).max() / sc
            for n in (2, 3, 4, 6)]
    assert errs[0] > errs[1] > 1e-15 or errs[1] < 1e-13
    assert errs[-1] < 1e-13


def test_reading_accuracy_against_exact():
    """The reading (exact double for cells closer than one in-plane edge,
    composite quadrature beyond) stays within 2e-13 of the largest component of
    the exact _Float128 tensor over random thin/thick layer pairs and offsets,
    while the plain double formula degrades with distance (the cancellation the
    reading exists for)."""
    rng = np.random.default_rng(1)
    worst_reading, worst_plain_far = 0.0, 0.0
    for _ in range(160):
        ti, tj = rng.uniform(0.3, 5.0, size=2)
        t, s = (2.0, 2.0, ti), (2.0, 2.0, tj)
        R = float(np.exp(rng.uniform(np.log(0.5), np.log(600.0))))
        d = rng.standard_normal(3)
        d[2] *= rng.uniform(0.01, 1.0)
        d *= R / np.linalg.norm(d)
        X, Y, Z = round(d[0] / 2) * 2.0, round(d[1] / 2) * 2.0, float(d[2])
        Nq = nw.tensor(X, Y, Z, t, s)
        sc = np.abs(Nq).max()
        worst_reading = max(worst_reading,
                            np.abs(nw.tensor(X, Y, Z, t, s, mode=nw.READING_D) - Nq).max() / sc)
        if R >= 300:
            worst_plain_far = max(worst_plain_far,
                                  np.abs(nw.tensor(X, Y, Z, t, s, mode=nw.EXACT_D) - Nq).max() / sc)
    assert worst_reading < 2e-13
    assert worst_plain_far > 1e-6


def test_layer_kernels_quadrant_parity():
    """The quadrant kernels expanded by the parity of N in the in-plane offsets
    (N_xx, N_yy, N_zz even; N_xy odd-odd; N_xz odd in X; N_yz odd in Y) equal
    the kernels evaluated directly at every offset."""
    from oracle import demag as dm
    th = [1.0, 0.5, 2.0]
    Kf = nw.layer_kernels(5, 4, 2.0, 2.0, th, mode=nw.READING_D, full=True)
    Kq = nw.layer_kernels(5, 4, 2.0, 2.0, th, mode=nw.READING_D, full=False)
    assert np.abs(dm.expand_quadrant(Kq) - Kf).max() < 1e-15
