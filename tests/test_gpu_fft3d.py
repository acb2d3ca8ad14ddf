"""GPU parity of the equidistant 3D-FFT method (Sec. 3.1, Eq. FFT_3D) through
the C ABI: demag_plan_create_equidistant + demag_apply against the oracle's
fft3d (z-offset kernels of the reading), the oracle's hybrid at equal
thicknesses and the GPU hybrid plan of the same stack.

Tolerances: 1e-11 relative L2 in double (as the hybrid's double path), 1e-5 in
float (the library's float bound: float FFTs along x, y and z)."""
import numpy as np
import pytest
import torch

import paper_1910_07054_gb300 as dm
from oracle import demag as odm
from paper_1910_07054_gb300 import inputs
from _cases import offset_kernels, reading_kernels, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _apply(plan, m_np, Ms, adjoint=False):
    m = torch.tensor(m_np, dtype=plan.dtype, device="cuda")
    H = torch.empty_like(m)
    if adjoint:
        dm.demag_apply_adjoint(plan.handle, m, Ms, H, info=plan.info)
    else:
        dm.demag_apply(plan.handle, m, Ms, H, info=plan.info)
    torch.cuda.synchronize()
    return H.double().cpu().numpy()


CASES = [
    (20, 12, 5, 0.7, 2),    # generic rows and columns, Pz = 16
    (9, 3, 1, 1.3, 1),      # one layer, Pz = 2
    (33, 17, 8, 0.5, 3),    # ragged, Pz = 16, L = Pz / 2
    (16, 16, 13, 2.0, 1),   # Pz = 32 with 13 layers
]


@pytest.mark.parametrize("nx,ny,nz,dz,B", CASES)
@pytest.mark.parametrize("prec,tol", [(dm.PREC_FP64, 1e-11), (dm.PREC_FP32, 1e-5)])
def test_equidistant_matches_oracle_fft3d(nx, ny, nz, dz, B, prec, tol):
    m = inputs.random_unit_vectors((B, nz, ny, nx), seed=nz + B)
    plan = dm.Plan.equidistant(nx, ny, nz, 2.0, 2.0, dz, precision=prec, max_batch=B)
    assert plan.info["path"] == 8 and plan.info["L"] == nz
    H = _apply(plan, m, 8e5)
    plan.close()
    assert dm.demag_wait_timeouts() == 0
    ref = odm.fft3d(offset_kernels(nx, ny, 2.0, 2.0, dz, nz), m, 8e5)
    assert rel_l2(H, ref) < tol
    # the hybrid of the same equal-thickness stack (Eq. FFT_v2) is the same field
    assert rel_l2(H, odm.hybrid(reading_kernels(nx, ny, 2.0, 2.0, (float(dz),) * nz), m, 8e5)) < tol


@pytest.mark.parametrize("nx,ny,nz", [(200, 140, 6), (20, 300, 4), (300, 11, 3)])
def test_equidistant_on_512_and_1024_point_transforms(nx, ny, nz):
    """Float plans whose rows or columns run the radix-8 512- and 1024-point
    kernels of the split path (Px = 512 / Py = 1024 / Px = 1024)."""
    m = inputs.random_unit_vectors((1, nz, ny, nx), seed=5)
    plan = dm.Plan.equidistant(nx, ny, nz, 2.0, 2.0, 1.5, precision=dm.PREC_FP32)
    H = _apply(plan, m, 1.0)
    plan.close()
    ref = odm.fft3d(offset_kernels(nx, ny, 2.0, 2.0, 1.5, nz), m, 1.0)
    assert rel_l2(H, ref) < 1e-5


def test_equidistant_agrees_with_the_hybrid_plan_and_is_self_adjoint():
    """256 x 256 cells, 24 layers of 1 nm: the 3D-FFT plan against the GPU hybrid
    plan of the same stack, and A^T = A (equal thicknesses: the adjoint's layer
    scales cancel)."""
    nx = ny = 256
    nz = 24
    m = inputs.random_unit_vectors((1, nz, ny, nx), seed=11)
    p3 = dm.Plan.equidistant(nx, ny, nz, 2.0, 2.0, 1.0, precision=dm.PREC_FP32)
    ph = dm.Plan(nx, ny, 2.0, 2.0, (1.0,) * nz, precision=dm.PREC_FP32)
    H3 = _apply(p3, m, 8e5)
    Hh = _apply(ph, m, 8e5)
    A3 = _apply(p3, m, 8e5, adjoint=True)
    p3.close()
    ph.close()
    assert rel_l2(H3, Hh) < 2e-6
    assert rel_l2(A3, H3) < 2e-6


def test_equidistant_tensor_structure():
    """The stored tensor at kz = 0 is the z-sum of the offset kernels' 2D
    spectra: its xz and yz parts (odd in z) vanish there, and the tensor has the
    documented size."""
    nx, ny, nz = 12, 10, 4
    plan = dm.Plan.equidistant(nx, ny, nz, 2.0, 2.0, 0.8, precision=dm.PREC_FP64)
    info = plan.info
    Kx, Qy, Qz = info["Px"] // 2 + 1, info["Py"] // 2 + 1, info["QyS"]
    assert Qz == 8 // 2 + 1
    T = torch.empty(Kx * Qy * Qz * 6, dtype=torch.float64, device="cuda")
    dm.demag_plan_tensor(plan.handle, T)
    torch.cuda.synchronize()
    plan.close()
    t = T.cpu().numpy().reshape(Kx, Qy, Qz, 6)
    assert np.abs(t[:, :, 0, 4:]).max() <= 1e-15 * np.abs(t).max()
    assert np.abs(t[:, :, Qz - 1, 4:]).max() <= 1e-13 * np.abs(t).max()  # kz = Pz/2: sin(pi r) = 0
    # kx = ky = kz = 0: the sum of every offset kernel, times 1/(Px Py Pz)
    Kz = offset_kernels(nx, ny, 2.0, 2.0, 0.8, nz)
    ref = Kz.sum(axis=(0, 2, 3)) / (info["Px"] * info["Py"] * 8)
    assert np.allclose(t[0, 0, 0, :4], ref[:4], rtol=1e-12, atol=1e-15)
