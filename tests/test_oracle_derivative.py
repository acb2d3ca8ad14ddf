"""Pins of the oracle's thickness derivatives (CPU).

The oracle differentiates the exact _Float128 tensor by central differences;
these tests tie that derivative to independent facts: the derivative of
Aharoni's prism closed form, the derivative of the dipole limit, the
additivity of thin slabs, and finite differences of the whole field.
"""
import math

import numpy as np
import pytest

from oracle import demag as odm
from oracle import newell as onw
from paper_1910_07054_gb300 import inputs
from test_oracle_newell import _aharoni_nzz


@pytest.mark.parametrize("edges", [(2.0, 2.0, 0.5), (1.0, 1.0, 1.0), (2.0, 3.0, 0.7)])
def test_self_term_thickness_derivative_matches_closed_form(edges):
    """Growing both cuboids of the self term together is d/dC of Aharoni's
    N_zz(A, B, C) (and of N_xx, N_yy by permutation)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    A, B, C = edges
    d = onw.tensor_dt(0, 0, 0, edges, edges, 1.0, 1.0, 0.0)

    def nzz(c):
        return _aharoni_nzz(A, B, float(c))

    ref_zz = mpmath.diff(lambda c: mpmath.mpf(nzz(c)), C, h=1e-4, method="step")
    ref_xx = mpmath.diff(lambda c: mpmath.mpf(_aharoni_nzz(B, float(c), A)), C, h=1e-4)
    assert d[2] == pytest.approx(float(ref_zz), abs=2e-7)
    assert d[0] == pytest.approx(float(ref_xx), abs=2e-7)
    assert d[:3].sum() == pytest.approx(0.0, abs=1e-14)  # the trace stays 1


def test_offset_derivative_matches_dipole_limit():
    """Far away dN/dZ tends to the Z-derivative of the point-dipole tensor."""
    t, s = (2.0, 2.0, 0.7), (2.0, 2.0, 1.9)
    X, Y, Z = 120.0, 80.0, 90.0

    def dip(Zc):
        c = np.array([X + (t[0] - s[0]) / 2, Y + (t[1] - s[1]) / 2, Zc + (t[2] - s[2]) / 2])
        r = np.linalg.norm(c)
        D = -(np.prod(s) / (4 * np.pi)) * (3 * np.outer(c, c) - r * r * np.eye(3)) / r ** 5
        return np.array([D[0, 0], D[1, 1], D[2, 2], D[0, 1], D[0, 2], D[1, 2]])

    h = 1e-3
    ref = (dip(Z + h) - dip(Z - h)) / (2 * h)
    d = onw.tensor_dt(X, Y, Z, t, s, 0.0, 0.0, 1.0)
    assert np.abs(d - ref).max() < 2e-3 * np.abs(ref).max()


@pytest.mark.parametrize("off", [(0.0, 0.0, 0.0), (2.0, -4.0, 1.0), (6.0, 2.0, -3.5)])
def test_source_edge_derivative_is_top_slab(off):
    """Additivity: a source of edge sz + e is the source of edge sz plus a slab
    of edge e on top, so dN/dsz = lim N(t <- slab e)(Z - sz) / e."""
    X, Y, Z = off
    t, s = (2.0, 2.0, 0.8), (2.0, 2.0, 1.3)
    d = onw.tensor_dt(X, Y, Z, t, s, 0.0, 1.0, 0.0)
    e = 1e-6
    slab = onw.tensor(X, Y, Z - s[2], t, (2.0, 2.0, e)) / e
    assert np.abs(d - slab).max() < 1e-5 * max(1.0, np.abs(d).max())


def test_field_derivative_matches_finite_differences():
    """dH/dt_l from the derivative kernels (linear in m) against a central
    difference of the whole oracle field with step 1e-3 nm."""
    nx, ny, th = 6, 5, np.array([1.0, 0.5, 2.0, 0.8])
    m = inputs.random_unit_vectors((len(th), ny, nx), seed=12)
    for layer in (0, 1, 3):
        dK = onw.layer_dkernels(nx, ny, 2.0, 2.0, th, layer)
        dH = odm.hybrid(dK, m, 1.0)
        h = 1e-3
        tp, tm = th.copy(), th.copy()
        tp[layer] += h
        tm[layer] -= h
        Hp = odm.hybrid(onw.layer_kernels(nx, ny, 2.0, 2.0, tp, mode=onw.EXACT_Q), m, 1.0)
        Hm = odm.hybrid(onw.layer_kernels(nx, ny, 2.0, 2.0, tm, mode=onw.EXACT_Q), m, 1.0)
        fd = (Hp - Hm) / (2 * h)
        assert np.linalg.norm(dH - fd) / np.linalg.norm(fd) < 1e-5
