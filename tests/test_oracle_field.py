"""Pins of the oracle's demagnetization field (Sec. 3) against independent routes.

* brute-force direct summation (Eq. Hi_discrete) vs the hybrid method (Eq. FFT_v2)
* equal thicknesses: hybrid vs the 3D-FFT method (Eq. FFT_3D)
* a stack of unequal layers vs the same stack cut into equal sub-layers and run
  through the 3D-FFT method with the classical (equal-cell) tensor
* a wide uniform film: H_z tends to -Ms, and equals -Ms N(cell <- film cuboid)
* the worked example of Sec. 4: optimum middle-layer thickness 3.44 nm
* volume-weighted self-adjointness of the field operator (reciprocity)
"""
import json
import os

import numpy as np
import pytest

from oracle import demag as dm
from oracle import newell as nw
from paper_1910_07054_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_direct_sum_equals_hybrid_quad_tensor():
    nx, ny = 7, 6
    th = [1.0, 0.5, 2.0]
    K = nw.layer_kernels(nx, ny, 2.0, 2.0, th, mode=nw.EXACT_Q, full=True)
    m = inputs.random_unit_vectors((2, 3, ny, nx), seed=3)
    Hd = dm.direct_sum(K, m, 8e5)
    Hh = dm.hybrid(K, m, 8e5)
    assert np.linalg.norm(Hh - Hd) / np.linalg.norm(Hd) < 1e-13


def test_hybrid_equals_3d_fft_for_equal_layers():
    nx, ny, L, t = 6, 5, 4, 0.7
    K = nw.layer_kernels(nx, ny, 2.0, 1.5, [t] * L, mode=nw.EXACT_Q, full=True)
    # with equal thicknesses N(i <- j) depends only on i - j
    Kz = np.stack([K[max(r, 0), max(-r, 0)] for r in range(-(L - 1), L)])
    for r in range(-(L - 1), L):
        for i in range(L):
            j = i - r
            if 0 <= j < L:
                assert np.abs(K[i, j] - Kz[r + L - 1]).max() < 1e-15
    m = inputs.random_unit_vectors((L, ny, nx), seed=4)
    H2 = dm.hybrid(K, m, 1.0)
    H3 = dm.fft3d(Kz, m, 1.0)
    assert np.linalg.norm(H2 - H3) / np.linalg.norm(H3) < 1e-13


def test_unequal_layers_equal_volume_averaged_equidistant_split():
    """Stack [1.0, 0.5, 2.0] nm equals an equidistant 0.5 nm stack of 2+1+4
    sub-layers (m constant within each original layer) once the sub-layer
    fields are volume-averaged back onto the original layers.  The split stack
    uses only equal cells (classical tensor) and the 3D FFT, so this checks the
    unequal-thickness generalization and the hybrid route together."""
    nx, ny = 6, 5
    th = [1.0, 0.5, 2.0]
    split = [2, 1, 4]
    Kh = nw.layer_kernels(nx, ny, 2.0, 2.0, th, mode=nw.EXACT_Q, full=True)
    m = inputs.random_unit_vectors((3, ny, nx), seed=5)
    Hh = dm.hybrid(Kh, m, 1.0)
    Ls = sum(split)
    Ks = nw.layer_kernels(nx, ny, 2.0, 2.0, [0.5] * Ls, mode=nw.EXACT_Q, full=True)
    Kz = np.stack([Ks[max(r, 0), max(-r, 0)] for r in range(-(Ls - 1), Ls)])
    ms = np.concatenate([np.repeat(m[l:l + 1], split[l], axis=0) for l in range(3)])
    Hs = dm.fft3d(Kz, ms, 1.0)
    start = np.cumsum([0] + split)
    Havg = np.stack([Hs[start[l]:start[l + 1]].mean(axis=0) for l in range(3)])
    assert np.linalg.norm(Hh - Havg) / np.linalg.norm(Havg) < 1e-12


def test_uniform_film_out_of_plane():
    """Uniform m = +z over a wide thin film: by additivity the centre cell's
    field is -Ms N_zz(cell <- whole film), and it tends to -Ms (an infinite
    film has H = -M_z) with a deviation of order thickness / width."""
    n, dx, t, Ms = 63, 2.0, 0.5, 8e5
    Kq = nw.layer_kernels(n, n, dx, dx, [t], mode=nw.READING_D, full=False)
    K = dm.expand_quadrant(Kq)
    m = np.zeros((1, 3, n, n))
    m[0, 2] = 1.0
    H = dm.hybrid(K, m, Ms)
    c = n // 2
    film = nw.tensor(c * dx, c * dx, 0.0, (dx, dx, t), (n * dx, n * dx, t))
    assert H[0, 2, c, c] == pytest.approx(-Ms * film[2], rel=1e-11)
    assert abs(H[0, 0, c, c]) < 1e-8 * Ms and abs(H[0, 1, c, c]) < 1e-8 * Ms
    assert abs(H[0, 2, c, c] / Ms + 1.0) < 2.0 * t / (n * dx)


def test_batch_equals_single_states():
    nx, ny, th = 5, 4, [0.9, 1.4]
    K = nw.layer_kernels(nx, ny, 2.0, 2.0, th, mode=nw.READING_D, full=True)
    m = inputs.random_unit_vectors((3, 2, ny, nx), seed=6)
    Hb = dm.hybrid(K, m, 2.0)
    for b in range(3):
        assert np.abs(Hb[b] - dm.hybrid(K, m[b], 2.0)).max() < 1e-14


def test_volume_weighted_self_adjoint():
    """sum_i t_i <u_i, (A v)_i> = sum_j t_j <(A u)_j, v_j> for the field operator
    A (reciprocity of the target-volume-normalised tensor)."""
    nx, ny, th = 6, 5, np.array([1.0, 0.5, 2.0])
    K = nw.layer_kernels(nx, ny, 2.0, 2.0, th, mode=nw.READING_D, full=True)
    u = inputs.random_unit_vectors((3, ny, nx), seed=7)
    v = inputs.random_unit_vectors((3, ny, nx), seed=8)
    Av, Au = dm.hybrid(K, v, 1.0), dm.hybrid(K, u, 1.0)
    lhs = np.einsum("l,lcyx,lcyx->", th, u, Av)
    rhs = np.einsum("l,lcyx,lcyx->", th, Au, v)
    assert lhs == pytest.approx(rhs, rel=1e-13)


def _safm_mean_hz(t):
    dx, th, m = inputs.safm_stack(t)
    Kq = nw.layer_kernels(64, 64, dx, dx, th, mode=nw.READING_D, full=False)
    H = dm.hybrid(dm.expand_quadrant(Kq), m, 1.0)
    return H[4, 2].mean()


@pytest.mark.slow
def test_safm_worked_example_optimum():
    """Sec. 4: Newton on the middle SAFM layer thickness, starting at 5 nm,
    drives the mean z-field over the free layer to zero at 3.44 nm."""
    with open(os.path.join(GOLDEN, "safm_example.json")) as fh:
        gold = json.load(fh)
    t = gold["initial_middle_nm"]
    for _ in range(8):
        f = _safm_mean_hz(t)
        h = 1e-3
        d = (_safm_mean_hz(t + h) - _safm_mean_hz(t - h)) / (2 * h)
        t -= f / d
        if abs(f) < 1e-9:
            break
    tol = 0.5 * 10.0 ** (-gold["printed_digits"])
    assert abs(t - gold["optimum_middle_nm"]) <= tol
    assert abs(_safm_mean_hz(t)) < 1e-8


def test_target_layer_hybrid_equals_full_hybrid():
    """The pair-by-pair restriction to selected target layers (used at sizes
    where all L x L kernels do not fit memory) is the same Eq. FFT_v2."""
    nx, ny, th = 6, 5, [1.0, 0.5, 2.0, 0.7]
    K = nw.layer_kernels(nx, ny, 2.0, 2.0, th, mode=nw.READING_D, full=True)
    m = inputs.random_unit_vectors((len(th), ny, nx), seed=14)
    H = dm.hybrid(K, m, 3.0)
    Ht = dm.hybrid_targets(lambda i, j: nw.pair_kernel(nx, ny, 2.0, 2.0, th, i, j), m, 3.0, [0, 3])
    assert np.abs(Ht[0] - H[0]).max() == 0.0 and np.abs(Ht[3] - H[3]).max() == 0.0
