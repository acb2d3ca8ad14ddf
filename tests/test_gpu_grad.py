"""GPU parity of the split column path, the adjoint (dH/dm) and the thickness
derivative (dH/dt_l), through the C ABI, against the oracle and against
central finite differences.

Tolerances: float64 fields within 1e-11 relative L2 of the oracle; the
derivative tensor within 1e-8 of its largest component (the closed form's
double-precision cancellation grows by one more power of distance / edge when
differentiated, and the quadrature switch sits at one in-plane edge of gap);
thickness gradients within 1e-6 relative of a central difference with step
1e-4 nm.
"""
import numpy as np
import pytest
import torch

import paper_1910_07054_gb300 as dm
from oracle import demag as odm
from oracle import newell as onw
from paper_1910_07054_gb300 import inputs
from paper_1910_07054_gb300.autograd import demag_field
from _cases import reading_kernels, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _field(plan, m_np, Ms, path=None):
    if path is not None:
        dm.demag_plan_set_path(plan.handle, path)
        plan.info = dm.demag_plan_info(plan.handle)
    m = torch.tensor(m_np, dtype=plan.dtype, device="cuda")
    H = plan.apply(m, Ms)
    torch.cuda.synchronize()
    return H.double().cpu().numpy()


def test_tensor_derivative_points_match_oracle():
    rng = np.random.default_rng(5)
    seeds = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, -1), (0, 1, 1), (0, 0, -1)]
    rows = []
    for k in range(140):
        ti, tj = rng.uniform(0.3, 5.0, size=2)
        R = float(np.exp(rng.uniform(np.log(0.5), np.log(400.0))))
        d = rng.standard_normal(3)
        d[2] *= rng.uniform(0.05, 1.0)
        d *= R / np.linalg.norm(d)
        X, Y, Z = round(d[0] / 2) * 2.0, round(d[1] / 2) * 2.0, float(d[2])
        rows.append([X, Y, Z, 2.0, 2.0, ti, 2.0, 2.0, tj, *seeds[k % len(seeds)]])
    # touching layers of a stack: Z = source edge (target right above the source)
    rows += [[0.0, 0.0, 0.9, 2.0, 2.0, 0.6, 2.0, 2.0, 0.9, 0, 1, 1],
             [4.0, 2.0, -0.6, 2.0, 2.0, 0.6, 2.0, 2.0, 0.6, 1, 0, 0],
             [0.0, 0.0, 0.0, 2.0, 2.0, 1.3, 2.0, 2.0, 1.3, 1, 1, 0]]
    g = np.array(rows)
    gt = torch.tensor(g, device="cuda")
    out = torch.empty(len(g), 6, dtype=torch.float64, device="cuda")
    dout = torch.empty_like(out)
    dm.demag_tensor_points_dt(gt, out, dout)
    torch.cuda.synchronize()
    N, dN = out.cpu().numpy(), dout.cpu().numpy()
    worst, where = 0.0, None
    for k, r in enumerate(g):
        ref = onw.tensor_dt(r[0], r[1], r[2], r[3:6], r[6:9], r[9], r[10], r[11])
        nref = onw.tensor(r[0], r[1], r[2], r[3:6], r[6:9])
        assert np.abs(N[k] - nref).max() < 5e-13 * np.abs(nref).max()
        sc = max(np.abs(ref).max(), 1e-300)
        err = np.abs(dN[k] - ref).max() / sc
        if err > worst:
            worst, where = err, r.tolist()
    assert worst < 1e-8, (worst, where)


CASES = [(20, 12, (1.0, 0.6, 2.0)), (16, 16, (0.5, 1.5, 0.5, 2.5, 1.0, 0.8, 3.0, 1.1)), (9, 3, (0.7, 1.2))]


@pytest.mark.parametrize("nx,ny,th", CASES)
@pytest.mark.parametrize("prec,tol", [(dm.PREC_FP64, 1e-13), (dm.PREC_FP32, 2e-6)])
def test_split_path_equals_fused_path(nx, ny, th, prec, tol):
    m = inputs.random_unit_vectors((2, len(th), ny, nx), seed=3)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=prec, max_batch=2)
    Hf = _field(plan, m, 1.0, path=1)
    Hs = _field(plan, m, 1.0, path=2)
    plan.close()
    assert rel_l2(Hs, Hf) < tol
    if prec == dm.PREC_FP64:
        K = reading_kernels(nx, ny, 2.0, 2.0, th)
        assert rel_l2(Hs, odm.hybrid(K, m, 1.0)) < 1e-11


def test_grad256_stack_fp64_matches_oracle():
    """256 x 256 x 10 layers, float64: more layers than the fused kernel holds in
    double, so the plan runs the split path."""
    c = inputs.CONFIGS["grad256"]
    th = tuple(inputs.thicknesses("grad256"))
    m = inputs.random_unit_vectors((len(th), c["ny"], c["nx"]), seed=0)
    plan = dm.Plan(c["nx"], c["ny"], c["dx"], c["dy"], th, precision=dm.PREC_FP64)
    assert plan.info["path"] == 2
    H = _field(plan, m[None], inputs.MS_DEFAULT)[0]
    plan.close()
    K = reading_kernels(c["nx"], c["ny"], c["dx"], c["dy"], th)
    assert rel_l2(H, odm.hybrid(K, m, inputs.MS_DEFAULT)) < 1e-11


def _adjoint(plan, g_np, Ms):
    g = torch.tensor(g_np, dtype=plan.dtype, device="cuda")
    out = torch.empty_like(g)
    dm.demag_apply_adjoint(plan.handle, g, Ms, out, info=plan.info)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("path", [1, 2])
def test_adjoint_matches_oracle_transposed_convolution(path):
    """A^T: the convolution with the transposed blocks N(j <- i)(-d)^T."""
    nx, ny, th = 11, 7, (1.0, 0.5, 2.0)
    g = inputs.random_unit_vectors((1, len(th), ny, nx), seed=9)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_FP64)
    dm.demag_plan_set_path(plan.handle, path)
    plan.info = dm.demag_plan_info(plan.handle)
    gm = _adjoint(plan, g, 3.0)[0]
    plan.close()
    K = reading_kernels(nx, ny, 2.0, 2.0, th)
    KT = np.transpose(K[:, :, :, ::-1, ::-1], (1, 0, 2, 3, 4))  # KT[i, j](d) = K[j, i](-d)
    assert rel_l2(gm, odm.hybrid(KT, g[0], 3.0)) < 1e-11


def test_adjoint_dot_product_identity():
    nx, ny = 64, 48
    th = tuple(inputs.thicknesses("grad256"))
    u = inputs.random_unit_vectors((1, len(th), ny, nx), seed=21)
    v = inputs.random_unit_vectors((1, len(th), ny, nx), seed=22)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_FP64)
    Av = _field(plan, v, 5.0)
    Atu = _adjoint(plan, u, 5.0)
    plan.close()
    lhs, rhs = float(np.sum(u * Av)), float(np.sum(Atu * v))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_dthickness_field_matches_oracle():
    nx, ny, th = 10, 8, np.array([1.0, 0.5, 2.0, 0.8])
    m = inputs.random_unit_vectors((1, len(th), ny, nx), seed=13)
    plan = dm.Plan(nx, ny, 2.0, 2.0, tuple(th), precision=dm.PREC_FP64)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda")
    for layer in (0, 2, 3):
        dH = torch.empty_like(mt)
        dm.demag_apply_dthickness(plan.handle, mt, 2.0, dH, layer, info=plan.info)
        torch.cuda.synchronize()
        ref = odm.hybrid(onw.layer_dkernels(nx, ny, 2.0, 2.0, th, layer), m[0], 2.0)
        assert rel_l2(dH[0].cpu().numpy(), ref) < 1e-9
    plan.close()


def _mean_free_hz(nx, ny, dx, th, m, Ms):
    plan = dm.Plan(nx, ny, dx, dx, tuple(th), precision=dm.PREC_FP64)
    H = _field(plan, m, Ms)
    plan.close()
    return H[0, -1, 2].mean()


def test_grad256_thickness_gradient_matches_central_differences():
    """d(mean H_z over the top layer)/d(thickness of layer 4, 1-based) on the
    256 x 256 x 10 stack, float64, against a central difference of step 1e-4 nm."""
    c = inputs.CONFIGS["grad256"]
    nx, ny, dx = c["nx"], c["ny"], c["dx"]
    th = inputs.thicknesses("grad256")
    L, layer, Ms = len(th), 3, inputs.MS_DEFAULT
    m = inputs.random_unit_vectors((1, L, ny, nx), seed=0)
    plan = dm.Plan(nx, ny, dx, dx, tuple(th), precision=dm.PREC_FP64)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda")
    gH = torch.zeros_like(mt)
    gH[0, -1, 2] = 1.0 / (nx * ny)
    g = dm.demag_thickness_grad(plan.handle, mt, gH, Ms, layer, info=plan.info)
    plan.close()
    h = 1e-4
    tp, tm = th.copy(), th.copy()
    tp[layer] += h
    tm[layer] -= h
    fd = (_mean_free_hz(nx, ny, dx, tp, m, Ms) - _mean_free_hz(nx, ny, dx, tm, m, Ms)) / (2 * h)
    assert abs(g - fd) <= 1e-6 * abs(fd)


def test_autograd_function_routes_both_gradients():
    nx, ny, th = 24, 16, [1.0, 0.6, 2.0, 0.9]
    m_np = inputs.random_unit_vectors((1, len(th), ny, nx), seed=31)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_FP64)
    m = torch.tensor(m_np, dtype=torch.float64, device="cuda", requires_grad=True)
    t = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    H = demag_field(m, t, plan, 8e5, layers=[1])
    loss = H[0, -1, 2].mean()
    loss.backward()
    gH = torch.zeros_like(m)
    gH[0, -1, 2] = 1.0 / (nx * ny)
    gm = torch.empty_like(m)
    dm.demag_apply_adjoint(plan.handle, gH.detach(), 8e5, gm, info=plan.info)
    g1 = dm.demag_thickness_grad(plan.handle, m.detach(), gH.detach(), 8e5, 1, info=plan.info)
    plan.close()
    assert torch.allclose(m.grad, gm, rtol=0, atol=1e-12 * gm.abs().max().item())
    assert t.grad[1].item() == pytest.approx(g1, rel=1e-12)
    assert t.grad[0].item() == 0.0 and t.grad[2].item() == 0.0


def test_adjoint_on_512_point_path():
    """The radix-8 512-point kernels carry the adjoint's layer scales
    (float64, 200 x 140 grid: 512-point rows and columns)."""
    nx, ny, th = 200, 140, (1.0, 0.5, 2.0)
    g = inputs.random_unit_vectors((1, len(th), ny, nx), seed=19)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_FP64)
    assert plan.info["path"] == 5
    gm = _adjoint(plan, g, 2.0)[0]
    plan.close()
    K = reading_kernels(nx, ny, 2.0, 2.0, th)
    KT = np.transpose(K[:, :, :, ::-1, ::-1], (1, 0, 2, 3, 4))
    assert rel_l2(gm, odm.hybrid(KT, g[0], 2.0)) < 1e-11


@pytest.mark.parametrize("nx,ny", [(200, 3), (3, 140)])
def test_dthickness_on_512_point_transforms(nx, ny):
    """The derivative tensor's full pair set through the 512-point row
    kernels (nx = 200) and the 512-point fused columns (ny = 140)."""
    th = np.array([1.0, 2.0])
    m = inputs.random_unit_vectors((1, len(th), ny, nx), seed=23)
    plan = dm.Plan(nx, ny, 2.0, 2.0, tuple(th), precision=dm.PREC_FP64)
    assert plan.info["path"] == (5 if ny == 140 else 1)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda")
    dH = torch.empty_like(mt)
    dm.demag_apply_dthickness(plan.handle, mt, 2.0, dH, 1, info=plan.info)
    torch.cuda.synchronize()
    plan.close()
    ref = odm.hybrid(onw.layer_dkernels(nx, ny, 2.0, 2.0, th, 1), m[0], 2.0)
    assert rel_l2(dH[0].cpu().numpy(), ref) < 1e-9


# ---- float plans ---------------------------------------------------------------
# The float kernels round every FFT stage and every contraction sum to float
# (unit roundoff 6e-8); over the log2(512) = 9 butterfly stages of each of the
# four transforms and the sum over L source layers the field carries a relative
# error of a few 1e-7 (4e-7 measured on the 256 x 256 x 8 stack).  The adjoint
# and the derivative field run the same kernels, so they are held to the float
# field's bound, 1e-5 relative L2.  The derivative tensor is built in double and
# stored in float (one more rounding per entry), which leaves that bound intact.
FLOAT_TOL = 1e-5


def _transposed_oracle(nx, ny, th, g, Ms):
    K = reading_kernels(nx, ny, 2.0, 2.0, tuple(th))
    KT = np.transpose(K[:, :, :, ::-1, ::-1], (1, 0, 2, 3, 4))  # KT[i, j](d) = K[j, i](-d)
    return odm.hybrid(KT, g, Ms)


@pytest.mark.parametrize("nx,ny,th,path", [
    (200, 140, (1.0, 0.5, 2.0), 5),        # 512-point rows and the streamed-ring columns
    (40, 24, (1.0, 0.6, 2.0, 0.9), 1),     # generic rows, fused columns
    (40, 24, (1.0, 0.6, 2.0, 0.9), 2),     # generic rows, split columns
])
def test_float_adjoint_matches_oracle_transposed_convolution(nx, ny, th, path):
    """A^T gH on float plans: the rows carry the source scales 1/t_j on input and
    the target scales t_i on output (Sec. 3 reciprocity), in float."""
    g = inputs.random_unit_vectors((1, len(th), ny, nx), seed=41)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_FP32)
    if path != 5:
        dm.demag_plan_set_path(plan.handle, path)
        plan.info = dm.demag_plan_info(plan.handle)
    assert plan.info["path"] == path
    gm = _adjoint(plan, g, 2.0)[0]
    plan.close()
    assert rel_l2(gm, _transposed_oracle(nx, ny, th, g[0], 2.0)) < FLOAT_TOL


def test_grad256_float_adjoint_matches_oracle():
    """The differentiation workload (256 x 256 x 10) on a float plan: the
    streamed-ring column kernel at 10 layers with the adjoint's layer scales."""
    c = inputs.CONFIGS["grad256"]
    th = tuple(inputs.thicknesses("grad256"))
    g = inputs.random_unit_vectors((1, len(th), c["ny"], c["nx"]), seed=43)
    plan = dm.Plan(c["nx"], c["ny"], c["dx"], c["dy"], th, precision=dm.PREC_FP32)
    assert plan.info["path"] == 5
    gm = _adjoint(plan, g, inputs.MS_DEFAULT)[0]
    plan.close()
    K = reading_kernels(c["nx"], c["ny"], c["dx"], c["dy"], th)
    KT = np.transpose(K[:, :, :, ::-1, ::-1], (1, 0, 2, 3, 4))
    assert rel_l2(gm, odm.hybrid(KT, g[0], inputs.MS_DEFAULT)) < FLOAT_TOL


@pytest.mark.parametrize("nx,ny,th,layers", [
    (10, 8, (1.0, 0.5, 2.0, 0.8), (0, 2, 3)),   # generic kernels
    (200, 3, (1.0, 2.0), (1,)),                 # 512-point row kernels
    (3, 140, (1.0, 2.0), (0, 1)),               # 512-point fused columns, all L^2 pairs
])
def test_float_dthickness_field_matches_oracle(nx, ny, th, layers):
    """dH/dt_l on float plans against the oracle's derivative kernels
    (_Float128 central differences of the exact tensor)."""
    th = np.array(th)
    m = inputs.random_unit_vectors((1, len(th), ny, nx), seed=47)
    plan = dm.Plan(nx, ny, 2.0, 2.0, tuple(th), precision=dm.PREC_FP32)
    mt = torch.tensor(m, dtype=torch.float32, device="cuda")
    for layer in layers:
        dH = torch.empty_like(mt)
        dm.demag_apply_dthickness(plan.handle, mt, 2.0, dH, layer, info=plan.info)
        torch.cuda.synchronize()
        ref = odm.hybrid(onw.layer_dkernels(nx, ny, 2.0, 2.0, th, layer), m[0], 2.0)
        assert rel_l2(dH[0].double().cpu().numpy(), ref) < FLOAT_TOL, layer
    plan.close()


def _oracle_mean_top_hz(nx, ny, dx, th, m, Ms):
    """Mean H_z of the top layer from the oracle (Eq. FFT_v2, target layer only,
    double-precision reading of the tensor)."""
    L = len(th)
    pk = lambda i, j: onw.pair_kernel(nx, ny, dx, dx, th, i, j)  # noqa: E731
    return odm.hybrid_targets(pk, m, Ms, [L - 1])[L - 1][2].mean()


def test_grad256_float_thickness_gradient_matches_oracle_central_difference():
    """d(mean H_z of the top layer)/d(thickness of layer 4, 1-based) on the
    256 x 256 x 10 stack from a float plan, against a central difference (step
    1e-4 nm) of the oracle's double-precision field.  The difference quotient
    carries the oracle's field error (~1e-13 relative) divided by the step, far
    below the float bound."""
    c = inputs.CONFIGS["grad256"]
    nx, ny, dx = c["nx"], c["ny"], c["dx"]
    th = inputs.thicknesses("grad256")
    L, layer, Ms = len(th), 3, inputs.MS_DEFAULT
    m = inputs.random_unit_vectors((1, L, ny, nx), seed=0)
    plan = dm.Plan(nx, ny, dx, dx, tuple(th), precision=dm.PREC_FP32)
    mt = torch.tensor(m, dtype=torch.float32, device="cuda")
    gH = torch.zeros_like(mt)
    gH[0, -1, 2] = 1.0 / (nx * ny)
    g = dm.demag_thickness_grad(plan.handle, mt, gH, Ms, layer, info=plan.info)
    plan.close()
    h = 1e-4
    tp, tm = th.copy(), th.copy()
    tp[layer] += h
    tm[layer] -= h
    fd = (_oracle_mean_top_hz(nx, ny, dx, tp, m[0], Ms) - _oracle_mean_top_hz(nx, ny, dx, tm, m[0], Ms)) / (2 * h)
    assert abs(g - fd) <= FLOAT_TOL * abs(fd), (g, fd)
