"""demag_apply_static, the entry point for callers that cannot allocate device
memory (for instance code running inside a framework whose allocator owns the
GPU's memory, or a time-critical loop that cannot afford the synchronisation an
allocation may bring).  It runs the demag_apply kernels with their workspace in
the library's fixed device array; its field must equal demag_apply's, call
after call, although every call reuses the same array.

This file is named to be collected last, so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest
import torch

import paper_1910_07054_gb300 as dm
from paper_1910_07054_gb300 import inputs

pytestmark = pytest.mark.gpu


def _stored_tensor(plan):
    info = plan.info
    n = (info["Px"] // 2 + 1) * info["npairs"] * 6 * info["QyS"]
    T = torch.empty(n, dtype=plan.dtype, device="cuda")
    dm.demag_plan_tensor(plan.handle, T)
    return T


@pytest.mark.parametrize("prec,tol", [(dm.PREC_FP32, 1e-5), (dm.PREC_FP64, 1e-11)])
def test_static_entry_matches_plan_apply_on_consecutive_calls(prec, tol):
    assert torch.cuda.is_available()
    nx, ny, th, Ms = 40, 24, (1.0, 0.5, 2.0, 0.8), 8e5
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=prec, max_batch=2)
    T = _stored_tensor(plan)
    for seed in (1, 2):  # two calls in a row, different states each time
        m = torch.tensor(inputs.random_unit_vectors((2, len(th), ny, nx), seed=seed),
                         dtype=plan.dtype, device="cuda")
        H_ref = plan.apply(m, Ms)
        H = torch.full_like(m, float("nan"))
        dm.demag_apply_static(T, th, nx, ny, prec, m, Ms, H)
        torch.cuda.synchronize()
        a, b = H.double().cpu().numpy(), H_ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < tol
    plan.close()


def test_static_entry_on_the_512_point_kernels():
    """256 x 256 x 8 float (the MRAM-like stack): radix-8 512-point rows and the
    streamed-ring column kernel with the tensor in natural folded-ky order, two
    calls in a row against demag_apply."""
    from paper_1910_07054_gb300.inputs import mram_magnetization
    c = inputs.CONFIGS["mram256"]
    th = tuple(float(t) for t in inputs.thicknesses("mram256"))
    nx, ny = c["nx"], c["ny"]
    plan = dm.Plan(nx, ny, c["dx"], c["dy"], th, precision=dm.PREC_FP32)
    assert plan.info["path"] == 5
    T = _stored_tensor(plan)
    for seed in (0, 1):
        m = torch.tensor(mram_magnetization(nx, ny, len(th), seed=seed, batch=1), dtype=torch.float32,
                         device="cuda")
        H_ref = plan.apply(m, inputs.MS_DEFAULT)
        H = torch.full_like(m, float("nan"))
        dm.demag_apply_static(T, th, nx, ny, dm.PREC_FP32, m, inputs.MS_DEFAULT, H)
        torch.cuda.synchronize()
        a, b = H.double().cpu().numpy(), H_ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5
    plan.close()


def test_static_entry_rejects_a_tensor_of_the_wrong_size():
    nx, ny, th = 40, 24, (1.0, 0.5, 2.0, 0.8)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_FP32)
    T = _stored_tensor(plan)
    plan.close()
    m = torch.zeros(1, 3, 3, ny, nx, dtype=torch.float32, device="cuda")  # 3 layers: another plan's size
    with pytest.raises(dm.DemagError) as ei:
        dm.demag_apply_static(T, th[:3], nx, ny, dm.PREC_FP32, m, 1.0, torch.empty_like(m))
    assert ei.value.status == 1
    assert "bytes" in str(ei.value)


def test_static_entry_rejects_requests_above_its_scratch():
    nx = ny = 512
    th = (1.0,) * 8
    T = torch.zeros(16, dtype=torch.float32, device="cuda")  # never read: rejected first
    m = torch.zeros(1, len(th), 3, ny, nx, dtype=torch.float32, device="cuda")
    with pytest.raises(dm.DemagError) as ei:
        dm.demag_apply_static(T, th, nx, ny, dm.PREC_FP32, m, 1.0, torch.empty_like(m))
    assert ei.value.status == 4
    assert "bytes of scratch" in str(ei.value)
