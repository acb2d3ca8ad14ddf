"""GPU tests of the micromagnetic relaxation (demag_relax_layer) through the C
ABI: the relaxed state against the oracle's effective field (no torque left),
its energy against the oracle's energy, the Stoner-Wohlfarth switching field of
a single cell (the astroid, a closed form), and the Sec. 4 MRAM hysteresis.

Tolerances: the relaxed torque, recomputed by the oracle from the oracle's own
demag field, below 1e-4 T (the relaxation's stopping torque is 1e-5 T; the
float plan's field differs from the oracle's by its float rounding); energies
within 1e-6 relative (1e-5 for float plans, whose demag fields carry ~1e-7
relative rounding); the single-cell switching field within one field step
(2 mT) plus 1 mT of the astroid value."""
import numpy as np
import pytest
import torch

import paper_1910_07054_gb300 as dm
from oracle import demag as odm
from oracle import micromag as omm
from oracle import newell as onw
from paper_1910_07054_gb300 import inputs
from paper_1910_07054_gb300 import micromag as pmm
from _cases import reading_kernels

pytestmark = pytest.mark.gpu

MU0 = 4e-7 * np.pi


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _oracle_fields(K, m, layer, Js):
    """b_self and b_bias (tesla) of layer `layer` from the oracle's hybrid."""
    other = m.copy()
    other[layer] = 0.0
    own = np.zeros_like(m)
    own[layer] = m[layer]
    Ms = Js / MU0
    b_bias = MU0 * odm.hybrid(K, other, Ms)[layer]
    b_self = MU0 * odm.hybrid(K, own, Ms)[layer]
    return b_self, b_bias


@pytest.mark.parametrize("prec", [dm.PREC_FP64, dm.PREC_FP32])
def test_relaxed_state_has_no_torque_in_the_oracle_field(prec):
    """A 24 x 20 disk layer between two pinned layers, relaxed from random
    directions in a tilted field: the oracle's effective field (its own energy
    terms, its own demag) leaves no torque on the result, and the library's
    energy equals the oracle's energy of that state."""
    nx, ny, th, layer = 24, 20, (2.0, 1.0, 1.5), 2
    dx = 1.5
    Js, A, Ku, b_ext = 1.2, 1.3e-11, 4e5, (0.05, -0.02, 0.2)
    mask = inputs.disk_mask(nx, ny)
    m = inputs.random_unit_vectors((len(th), ny, nx), seed=8)
    m[0] = 0.0
    m[0, 2][mask] = 1.0
    m[1] = 0.0
    m[layer] *= mask
    plan = dm.Plan(nx, ny, dx, dx, th, precision=prec)
    mt = torch.tensor(m, dtype=plan.dtype, device="cuda")
    mk = torch.tensor(mask.astype(np.uint8), device="cuda")
    st = dm.demag_relax_layer(plan.handle, mt, layer, mk, Js, A, Ku, b_ext, tol_torque=1e-5, max_iter=5000,
                              info=plan.info)
    plan.close()
    assert st["converged"] in (1, 2) and st["max_torque"] < 1e-4
    mr = mt.double().cpu().numpy()
    assert np.array_equal(mr[:layer], m[:layer])  # pinned layers untouched
    assert np.allclose(np.linalg.norm(mr[layer], axis=0)[mask], 1.0, atol=1e-6)
    K = reading_kernels(nx, ny, dx, dx, th)
    b_self, b_bias = _oracle_fields(K, mr, layer, Js)
    L = 1e-9
    b = omm.effective_field(mr[layer], mask, dx * L, dx * L, Js, A, Ku, b_ext, b_self, b_bias)
    torque = np.linalg.norm(np.cross(mr[layer], b, axis=0), axis=0)[mask]
    assert torque.max() < 1e-4
    E = omm.energy(mr[layer], mask, dx * L, dx * L, th[layer] * L, Js, A, Ku, b_ext, b_self, b_bias)
    assert st["energy"] == pytest.approx(E, rel=1e-6 if prec == dm.PREC_FP64 else 1e-5)


def test_single_cell_switching_field_is_the_stoner_wohlfarth_astroid():
    """One 2 x 2 x 1 nm cell (uniform by construction) with uniaxial anisotropy
    along z, field applied 10 degrees off the axis: the magnetization leaves the
    +z branch at b = H_K / (cos^(2/3) psi + sin^(2/3) psi)^(3/2), with
    H_K = 2 Ku mu0 / Js - Js (N_zz - N_xx) and N the cell's self term."""
    Js, Ku, psi = 1.75, 2.09e6, 10.0
    N = onw.tensor(0.0, 0.0, 0.0, (2.0, 2.0, 1.0), (2.0, 2.0, 1.0))
    HK = 2 * Ku * MU0 / Js - Js * (N[2] - N[0])
    r = np.radians(psi)
    b_sw = HK / (np.cos(r) ** (2 / 3) + np.sin(r) ** (2 / 3)) ** 1.5
    plan = dm.Plan(1, 1, 2.0, 2.0, (1.0,), precision=dm.PREC_FP64)
    m = torch.zeros(1, 3, 1, 1, dtype=torch.float64, device="cuda")
    m[0, 2] = 1.0
    step = 2e-3
    bs = np.arange(0.0, -(b_sw + 0.05), -step)
    loop = pmm.hysteresis(plan, m, 0, np.ones((1, 1), bool), bs, Js=Js, A_ex=0.0, Ku=Ku, tilt_deg=psi,
                          tol_torque=1e-9, stop_after_switch=1)
    plan.close()
    found = pmm.switching_field(loop)
    assert found is not None
    assert b_sw - 1e-3 <= found <= b_sw + step + 1e-3, (found, b_sw)


def test_mram_free_layer_hysteresis_switches():
    """The Sec. 4 stack (64 x 64 cells over the 60 nm disk, layers [5, 1, 3.44, 1,
    3] nm, SAFM pinned, CoFe free layer): sweeping the field along z from +2 T
    down, the free layer stays on the +z branch through zero field (remanence)
    and switches to -z at a field between the uniform-rotation bound of a thin
    disk and the anisotropy field 2 Ku mu0 / Js = 3.0 T."""
    dx, th, m, mask, layer = pmm.mram_stack()
    plan = dm.Plan(64, 64, dx, dx, th, precision=dm.PREC_FP32)
    mt = torch.tensor(m, dtype=torch.float32, device="cuda")
    bs = np.arange(2.0, -3.2, -0.02)
    loop = pmm.hysteresis(plan, mt, layer, mask, bs, tol_torque=1e-4, stop_after_switch=2)
    plan.close()
    at_zero = [mz for b, mz, _, _ in loop if abs(b) < 1e-9]
    assert at_zero and at_zero[0] > 0.99
    b_sw = pmm.switching_field(loop)
    assert b_sw is not None and 0.5 < b_sw < 2 * pmm.KU_COFE * MU0 / pmm.JS_COFE
    assert loop[-1][1] < -0.9
