"""GPU parity of the batched, many-layer contraction (DEMAG_PREC_SPLIT_TF32 and
DEMAG_PREC_SPLIT_BF16): the dense-product contraction on the tcgen05 tensor
cores (three TF32 passes, path 6, or three BF16 passes, path 7), with
warp-level MMAs (path 4) and the same products on the FP32 cores (path 3),
against the oracle.

Tolerance: 1e-5 relative L2 against the float64 oracle for all (the
library's float32 target); the TF32 variants within 3e-6 of each other.  The
BF16 split keeps 16 significant bits of each operand (hi and lo of 8 each) and
drops lo x lo: each product is within about 3 x 2^-18 = 1.1e-5 of exact, and
with errors of random sign over the sum the field comes out near 2e-6 (a
float64 emulation of the split on 16 x 16 x 64 and 32 x 32 x 16 stacks gave
2.25e-6); it is held to the same 1e-5 against the oracle and the FP32 cores.
"""
import numpy as np
import pytest
import torch

import paper_1910_07054_gb300 as dm
from oracle import demag as odm
from oracle import newell as onw
from paper_1910_07054_gb300 import inputs
from _cases import reading_kernels, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _fields(plan, m, Ms, paths):
    out = {}
    mt = torch.tensor(m, dtype=torch.float32, device="cuda")
    for path in paths:
        dm.demag_plan_set_path(plan.handle, path)
        plan.info = dm.demag_plan_info(plan.handle)
        H = plan.apply(mt, Ms)
        torch.cuda.synchronize()
        out[path] = H.double().cpu().numpy()
    return out


@pytest.mark.parametrize("nx,ny,th,B", [
    (48, 40, tuple(np.round(np.linspace(0.5, 3.0, 16), 3)), 8),   # tiles without padding
    (21, 13, (1.0, 0.5, 2.0, 0.8, 1.7), 3),                        # L and B padded
    (32, 32, tuple(np.round(np.linspace(2.5, 0.6, 32), 3)), 16),
    (24, 20, tuple(np.round(np.linspace(0.7, 2.9, 10), 3)), 4),    # layers padded to 16, one row tile
    (17, 12, tuple(np.round(np.linspace(3.0, 0.5, 50), 3)), 6),    # layers padded to 56, two row tiles
    (20, 300, (1.0, 0.5, 2.0, 0.8), 2),                            # Py = 1024 columns, ragged ny
    (9, 512, (1.2, 0.7, 2.5), 3),                                  # Py = 1024 columns, ny = 512, odd L
    (300, 11, (1.0, 0.5, 2.0, 0.8), 2),                            # Px = 1024 rows, ragged nx, odd ny
])
def test_split_tf32_matches_oracle(nx, ny, th, B):
    m = inputs.random_unit_vectors((B, len(th), ny, nx), seed=len(th) + B)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_SPLIT_TF32, max_batch=B)
    even = len(th) % 2 == 0
    assert plan.info["path"] == (6 if even else 4)  # tcgen05 (path 6) wherever it holds the plan
    dm.demag_plan_set_path(plan.handle, 3)
    dm.demag_plan_set_path(plan.handle, 0)  # back to the default
    assert dm.demag_plan_info(plan.handle)["path"] == (6 if even else 4)
    paths = (4, 3, 6, 7) if even else (4, 3)
    H = _fields(plan, m, 8e5, paths)
    plan.close()
    assert dm.demag_wait_timeouts() == 0
    K = reading_kernels(nx, ny, 2.0, 2.0, th)
    ref = odm.hybrid(K, m, 8e5)
    for p in paths:
        assert rel_l2(H[p], ref) < 1e-5, p
        assert rel_l2(H[p], H[3]) < (1e-5 if p == 7 else 3e-6), p


def test_scale512_batch_sampled_against_oracle():
    """512 x 512 cells, 64 layers, 16 states: both contraction variants agree at
    full size, and one target layer of one state is checked against the oracle
    (computed pair by pair)."""
    c = inputs.CONFIGS["scale512"]
    nx, ny, B = c["nx"], c["ny"], c["batch"]
    th = inputs.thicknesses("scale512")
    L = len(th)
    m = inputs.random_unit_vectors((B, L, ny, nx), seed=0)
    plan = dm.Plan(nx, ny, c["dx"], c["dy"], tuple(th), precision=dm.PREC_SPLIT_TF32, max_batch=B)
    H = _fields(plan, m, inputs.MS_DEFAULT, (4, 3, 6, 7))
    plan.close()
    assert dm.demag_wait_timeouts() == 0
    assert rel_l2(H[4], H[3]) < 3e-6
    assert rel_l2(H[6], H[3]) < 3e-6
    assert rel_l2(H[7], H[3]) < 1e-5
    target, state = 37, 5
    ref = odm.hybrid_targets(lambda i, j: onw.pair_kernel(nx, ny, c["dx"], c["dy"], th, i, j),
                             m[state], inputs.MS_DEFAULT, [target])[target]
    assert rel_l2(H[4][state, target], ref) < 1e-5
    assert rel_l2(H[3][state, target], ref) < 1e-5
    assert rel_l2(H[6][state, target], ref) < 1e-5
    assert rel_l2(H[7][state, target], ref) < 1e-5


@pytest.mark.parametrize("path,nx,ny", [(3, 13, 9), (4, 13, 9), (6, 13, 9), (6, 290, 270), (7, 13, 9),
                                        (7, 290, 270)])
def test_split_tf32_adjoint_matches_oracle(path, nx, ny):
    """The adjoint (transposed-block convolution) through the dense-product
    contraction: sources scaled by 1/t_j and targets by t_i around the same
    products (290 x 270: the scales inside the 1024-point row kernels)."""
    th, B = (1.0, 0.5, 2.0, 0.8), 3
    g = inputs.random_unit_vectors((B, len(th), ny, nx), seed=31)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_SPLIT_TF32, max_batch=B)
    dm.demag_plan_set_path(plan.handle, path)
    info = dm.demag_plan_info(plan.handle)
    gt = torch.tensor(g, dtype=torch.float32, device="cuda")
    out = torch.empty_like(gt)
    dm.demag_apply_adjoint(plan.handle, gt, 3.0, out, info=info)
    torch.cuda.synchronize()
    plan.close()
    assert dm.demag_wait_timeouts() == 0
    K = reading_kernels(nx, ny, 2.0, 2.0, th)
    KT = np.transpose(K[:, :, :, ::-1, ::-1], (1, 0, 2, 3, 4))  # KT[i, j](d) = K[j, i](-d)
    assert rel_l2(out.double().cpu().numpy(), odm.hybrid(KT, g, 3.0)) < 1e-5


def test_split_bf16_plan_defaults_to_the_bf16_tcgen05_path():
    """A DEMAG_PREC_SPLIT_BF16 plan runs path 7 by default (even L <= 64, B <= 16)
    and falls back to the warp-level TF32 MMAs (path 4) elsewhere; both stay
    within the float bound of the oracle."""
    for nx, ny, th, B, path in ((40, 36, tuple(np.round(np.linspace(0.6, 2.4, 12), 3)), 5, 7),
                                (30, 20, (1.0, 0.5, 2.0), 2, 4)):
        m = inputs.random_unit_vectors((B, len(th), ny, nx), seed=7)
        plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_SPLIT_BF16, max_batch=B)
        assert plan.info["path"] == path and plan.info["precision"] == dm.PREC_SPLIT_BF16
        H = plan.apply(torch.tensor(m, dtype=torch.float32, device="cuda"), 8e5)
        torch.cuda.synchronize()
        plan.close()
        ref = odm.hybrid(reading_kernels(nx, ny, 2.0, 2.0, th), m, 8e5)
        assert rel_l2(H.double().cpu().numpy(), ref) < 1e-5


def test_bf16_plan_equals_tf32_plan_on_path_7_bit_for_bit():
    """Path 7 splits every tensor value into BF16 hi + lo: a DEMAG_PREC_SPLIT_TF32
    plan in the kernel, from its float tensor, a DEMAG_PREC_SPLIT_BF16 plan at
    plan time, storing the pairs with N_zz negated.  The operands and so the
    fields are the same, bit for bit.  Compressed, the two plans judge a block
    by its float value and by hi + lo (within 2^-18 of it), which may part at
    the tolerance's edge: the fields agree to 1e-6.  The BF16 plan runs path 7
    only."""
    nx, ny, B = 40, 36, 3
    th = tuple(np.round(np.linspace(0.6, 2.4, 12), 3))
    m = torch.tensor(inputs.random_unit_vectors((B, len(th), ny, nx), seed=23), dtype=torch.float32, device="cuda")
    p32 = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_SPLIT_TF32, max_batch=B)
    p16 = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_SPLIT_BF16, max_batch=B)
    try:
        dm.demag_plan_set_path(p32.handle, 7)
        assert p16.info["path"] == 7
        for path in (3, 4, 6):
            with pytest.raises(dm.DemagError):
                dm.demag_plan_set_path(p16.handle, path)
        assert torch.equal(p32.apply(m, 8e5), p16.apply(m, 8e5))
        g32 = torch.empty_like(m)
        g16 = torch.empty_like(m)
        dm.demag_apply_adjoint(p32.handle, m, 3.0, g32, info=p32.info)
        dm.demag_apply_adjoint(p16.handle, m, 3.0, g16, info=p16.info)
        assert torch.equal(g32, g16)
        p32.compress(1e-8)
        p16.compress(1e-8)
        h32, h16 = p32.apply(m, 8e5), p16.apply(m, 8e5)
        assert float(torch.linalg.vector_norm(h32 - h16) / torch.linalg.vector_norm(h32)) < 1e-6
        torch.cuda.synchronize()
        assert dm.demag_wait_timeouts() == 0
    finally:
        p32.close()
        p16.close()


@pytest.mark.parametrize("prec,nx,ny,th,shrinks", [
    (dm.PREC_SPLIT_BF16, 64, 48, tuple(np.round(np.linspace(0.6, 2.4, 20), 3)), False),
    (dm.PREC_SPLIT_TF32, 40, 36, tuple(np.round(np.linspace(0.5, 3.0, 24), 3)), False),
    (dm.PREC_SPLIT_BF16, 32, 24, (1.0,) * 8 + (100.0, 100.0) + (1.0,) * 8, True),
    (dm.PREC_SPLIT_BF16, 13, 9, (1.0, 0.5, 2.0, 0.8), False),
])
def test_compressed_tensor_field_and_adjoint_match_oracle(prec, nx, ny, th, shrinks):
    """demag_plan_compress drops the 8 x 8 layer blocks below 1e-8 of their
    component's maximum; the field and the adjoint of the compressed plan stay
    within the float bound of the oracle.  The stack with two 100 nm spacer
    layers puts its last block 200 nm above the first, so that block pair
    drops at all but the lowest in-plane frequencies."""
    B = 3
    m = inputs.random_unit_vectors((B, len(th), ny, nx), seed=17)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=prec, max_batch=B)
    full = plan.info
    nb = (len(th) + 7) // 8
    full_bytes = (full["Px"] // 2 + 1) * (full["Py"] // 2 + 1) * 6 * 64 * nb * (nb + 1) // 2 * 4
    stored = plan.compress(1e-8)
    assert 0 < stored <= full_bytes
    if shrinks:
        assert stored < 0.95 * full_bytes, (stored, full_bytes)
    mt = torch.tensor(m, dtype=torch.float32, device="cuda")
    H = plan.apply(mt, 8e5)
    out = torch.empty_like(mt)
    dm.demag_apply_adjoint(plan.handle, mt, 3.0, out, info=plan.info)
    torch.cuda.synchronize()
    plan.close()
    assert dm.demag_wait_timeouts() == 0
    K = reading_kernels(nx, ny, 2.0, 2.0, th)
    assert rel_l2(H.double().cpu().numpy(), odm.hybrid(K, m, 8e5)) < 1e-5
    KT = np.transpose(K[:, :, :, ::-1, ::-1], (1, 0, 2, 3, 4))
    assert rel_l2(out.double().cpu().numpy(), odm.hybrid(KT, m, 3.0)) < 1e-5


def test_compressed_plan_restrictions():
    """After compression only paths 6 and 7 run and the tensor is not exported;
    a second compression, other precisions and a bad tolerance are refused."""
    th = (1.0, 0.5, 2.0, 0.8)
    plan = dm.Plan(12, 10, 2.0, 2.0, th, precision=dm.PREC_SPLIT_TF32, max_batch=2)
    try:
        with pytest.raises(dm.DemagError):
            plan.compress(-1.0)
        with pytest.raises(dm.DemagError):
            plan.compress(1.0)
        plan.compress(0.0)
        with pytest.raises(dm.DemagError):
            plan.compress(1e-8)
        for path in (3, 4):
            with pytest.raises(dm.DemagError):
                dm.demag_plan_set_path(plan.handle, path)
        for path in (6, 7, 0):
            dm.demag_plan_set_path(plan.handle, path)
        with pytest.raises(dm.DemagError):
            dm.demag_plan_tensor(plan.handle, torch.empty(16, dtype=torch.float32, device="cuda"))
    finally:
        plan.close()
    p32 = dm.Plan(12, 10, 2.0, 2.0, th, precision=dm.PREC_FP32)
    try:
        with pytest.raises(dm.DemagError):
            p32.compress(1e-8)
    finally:
        p32.close()
