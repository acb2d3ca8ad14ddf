"""Failure handling without a GPU fault: a host-side injected allocation failure
and the bounded device wait of the streamed column kernel, made to run out on
purpose by a barrier that nothing completes (a short limit; the kernel returns
normally and the host reads the count)."""
import numpy as np
import pytest
import torch

import paper_1910_07054_gb300 as dm
from paper_1910_07054_gb300 import inputs
from paper_1910_07054_gb300._lib import DEMAG_ENOMEM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    dm.demag_debug_fail_alloc(-1)
    torch.cuda.synchronize()


def _field(plan, m):
    H = plan.apply(torch.tensor(m, dtype=plan.dtype, device="cuda"), 1.0)
    torch.cuda.synchronize()
    return H.cpu().numpy()


def test_injected_allocation_failure_is_reported_and_recovered():
    th = (1.0, 0.5, 2.0)
    m = inputs.random_unit_vectors((1, len(th), 12, 20), seed=3)
    ref_plan = dm.Plan(20, 12, 2.0, 2.0, th, precision=dm.PREC_FP64)
    ref = _field(ref_plan, m)
    ref_plan.close()
    failed = 0
    for after in range(0, 16):
        dm.demag_debug_fail_alloc(after)
        try:
            plan = dm.Plan(20, 12, 2.0, 2.0, th, precision=dm.PREC_FP64)
        except dm.DemagError as e:
            assert e.status == DEMAG_ENOMEM
            assert "demag_debug_fail_alloc" in str(e)
            failed += 1
        else:
            plan.close()
        dm.demag_debug_fail_alloc(-1)
    assert failed >= 5  # every allocation of plan creation and tensor build was refused once
    plan = dm.Plan(20, 12, 2.0, 2.0, th, precision=dm.PREC_FP64)
    assert np.array_equal(_field(plan, m), ref)
    plan.close()


def test_injected_failure_in_a_lazy_workspace():
    th = (1.0, 0.5)
    m = torch.tensor(inputs.random_unit_vectors((1, 2, 8, 10), seed=4), dtype=torch.float64, device="cuda")
    plan = dm.Plan(10, 8, 2.0, 2.0, th, precision=dm.PREC_FP64)
    gH = torch.ones_like(m)
    dm.demag_debug_fail_alloc(0)  # the derivative workspace is allocated on first use
    with pytest.raises(dm.DemagError) as ei:
        dm.demag_thickness_grad(plan.handle, m, gH, 1.0, 0, info=plan.info)
    assert ei.value.status == DEMAG_ENOMEM
    dm.demag_debug_fail_alloc(-1)
    g = dm.demag_thickness_grad(plan.handle, m, gH, 1.0, 0, info=plan.info)
    assert np.isfinite(g)
    plan.close()


def test_bounded_wait_gives_up_and_is_reported():
    assert dm.demag_wait_timeouts() == 0
    dm.demag_selftest_bounded_wait(1 << 20)
    assert dm.demag_wait_timeouts() == 1
    assert dm.demag_wait_timeouts() == 0  # reading clears the count
    with pytest.raises(dm.DemagError):
        dm.demag_selftest_bounded_wait(0)


def test_synchronising_call_reports_a_timeout_as_an_error():
    """A bounded wait that gave up (here the self test's, with a short limit)
    makes the next synchronising entry point return DEMAG_ECUDA instead of a
    silently invalid field; the report is taken once, so the call after it
    succeeds and demag_wait_timeouts has nothing left to report."""
    from paper_1910_07054_gb300._lib import DEMAG_ECUDA
    th = (1.0, 0.5)
    m = inputs.random_unit_vectors((1, 2, 12, 20), seed=5).astype(np.float32)
    plan = dm.Plan(20, 12, 2.0, 2.0, th, precision=dm.PREC_FP32)
    mh = torch.tensor(m).pin_memory()
    Hh = torch.empty_like(mh).pin_memory()
    dm.demag_apply_host(plan.handle, mh, 1.0, Hh, info=plan.info)
    ref = Hh.clone()
    assert dm.demag_wait_timeouts() == 0
    dm.demag_selftest_bounded_wait(1 << 16)
    with pytest.raises(dm.DemagError) as ei:
        dm.demag_apply_host(plan.handle, mh, 1.0, Hh, info=plan.info)
    assert ei.value.status == DEMAG_ECUDA
    assert "bounded device wait" in str(ei.value)
    Hh.zero_()
    dm.demag_apply_host(plan.handle, mh, 1.0, Hh, info=plan.info)
    assert torch.equal(Hh, ref)
    assert dm.demag_wait_timeouts() == 0
    dm.demag_selftest_bounded_wait(1 << 16)
    mt = mh.cuda()
    with pytest.raises(dm.DemagError) as ei:
        dm.demag_apply_timed(plan.handle, mt, 1.0, torch.empty_like(mt), info=plan.info)
    assert ei.value.status == DEMAG_ECUDA
    plan.close()
