"""GPU tests of the surrogate network kernels and of the surrogate-assisted
thickness optimisation (Sec. 4).

Kernels: forward and backward against the float64 oracle network with the same
bfloat16 weights (float accumulation: 1e-5 relative on outputs, 1e-4 on
gradients); one Adam step against torch.optim.Adam on the CPU.
Optimisation: on the Sec. 4-like stack the surrogate, trained on solver
samples by these kernels, must reach the exact optimum of the design
thickness within 1e-3 nm with fewer exact solves than exact Newton.
"""
import numpy as np
import pytest
import torch

import paper_1910_07054_gb300 as dm
from oracle import mlp as omlp
from paper_1910_07054_gb300 import inputs
from paper_1910_07054_gb300 import surrogate as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _bf16_weights(I, H, O, seed):
    vals, bits = inputs.bf16_round(inputs.mlp_init(I, H, O, seed) * 3.0)
    wb = torch.from_numpy(bits.view(np.int16)).to("cuda").view(torch.bfloat16)
    return vals.astype(np.float64), wb


@pytest.mark.parametrize("I,H,O,N", [(8, 64, 3, 77), (5, 20, 2, 32), (1, 3, 1, 1)])
def test_mlp_kernels_match_oracle(I, H, O, N):
    w, wb = _bf16_weights(I, H, O, seed=I + H)
    rng = np.random.default_rng(N)
    x = rng.standard_normal((N, I)).astype(np.float32)
    gy = rng.standard_normal((N, O)).astype(np.float32)
    xt = torch.tensor(x, device="cuda")
    y = torch.empty(N, O, device="cuda")
    dm.demag_mlp_forward(wb, xt, y, I, H, O)
    gw = torch.zeros(dm.demag_mlp_param_count(I, H, O), device="cuda")
    gx = torch.empty_like(xt)
    dm.demag_mlp_backward(wb, xt, torch.tensor(gy, device="cuda"), gw, gx, I, H, O)
    torch.cuda.synchronize()
    y_ref, _ = omlp.forward(w, x, I, H, O)
    gw_ref, gx_ref = omlp.backward(w, x, gy, I, H, O)
    assert np.abs(y.cpu().numpy() - y_ref).max() <= 1e-5 * np.abs(y_ref).max()
    assert np.abs(gw.cpu().numpy() - gw_ref).max() <= 1e-4 * np.abs(gw_ref).max()
    assert np.abs(gx.cpu().numpy() - gx_ref).max() <= 1e-4 * np.abs(gx_ref).max()


def test_adam_step_matches_torch():
    P = 1000
    rng = np.random.default_rng(2)
    w0 = rng.standard_normal(P).astype(np.float32)
    g0 = rng.standard_normal(P).astype(np.float32)
    w = torch.tensor(w0, device="cuda")
    wb = torch.empty(P, dtype=torch.bfloat16, device="cuda")
    m1 = torch.zeros_like(w)
    m2 = torch.zeros_like(w)
    wr = torch.tensor(w0, requires_grad=True)
    opt = torch.optim.Adam([wr], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for step in (1, 2, 3):
        g = torch.tensor(g0 * step, device="cuda")
        dm.demag_mlp_adam(w, wb, g, m1, m2, 1e-2, 0.9, 0.999, 1e-8, step)
        wr.grad = torch.tensor(g0 * step)
        opt.step()
        assert float(g.abs().max()) == 0.0
    torch.cuda.synchronize()
    assert np.abs(w.cpu().numpy() - wr.detach().numpy()).max() < 1e-6
    assert torch.equal(wb.cpu(), w.cpu().to(torch.bfloat16))


def test_layer_mean_kernel():
    H = torch.randn(2, 4, 3, 9, 7, dtype=torch.float64, device="cuda")
    out = torch.empty(2, 3, dtype=torch.float64, device="cuda")
    dm.demag_layer_mean(H, dm.PREC_FP64, 2, out)
    assert torch.allclose(out, H[:, 2].mean(dim=(-1, -2)), rtol=1e-13, atol=1e-15)


def test_surrogate_newton_needs_fewer_exact_solves():
    """Sec. 4-like stack on a 64 x 64 grid (2 nm cells): train on solver
    samples, then optimise the layer-5 thickness from 5 nm."""
    solver = sg.ExactSolver(64, 2.0)
    T = inputs.opt_samples(600, seed=0)
    T, Y = sg.generate_samples(solver, T)
    net = sg.Surrogate(seed=0)
    hist = net.fit(T[:500], Y[:500], steps=3000, lr=3e-3)
    assert hist[-1][1] < 1e-3
    held = net.predict(T[500:])[:, 2]
    assert np.sqrt(np.mean((held - Y[500:, 2]) ** 2)) < 0.05 * np.abs(Y[:, 2]).max()

    t0 = inputs.OPT_BASE.copy()
    solver.solves = 0
    exact = sg.newton_exact(solver, t0, tol=1e-7)
    t_star = exact[-1][0]
    n_exact = next(s for (t, hz, s) in exact if abs(t - t_star) < 1e-3)
    solver.solves = 0
    sur = sg.newton_surrogate(solver, net, t0, tol=1e-7)
    n_sur = next(s for (t, hz, s, kind) in sur if abs(t - t_star) < 1e-3)
    assert abs(sur[-1][0] - t_star) < 1e-3
    assert n_sur < n_exact, (n_sur, n_exact, exact, sur)


@pytest.fixture(scope="module")
def _samples_256():
    solver = sg.ExactSolver(256, 2.0)
    T, Y = sg.generate_samples(solver, inputs.opt_samples(2000, seed=0))
    return solver, T, Y


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_surrogate_newton_needs_fewer_exact_solves_at_256(_samples_256, seed):
    """The same optimisation on the 256 x 256 x 8 stack of the optimisation
    workload (2000 solver samples, layer 5 in [0.5, 5] nm, the others +-10 %):
    for each of three trainings the surrogate-proposed Newton steps reach the
    optimum within 1e-3 nm in fewer exact solves than exact Newton."""
    solver, T, Y = _samples_256
    net = sg.Surrogate(seed=seed)
    hist = net.fit(T[:1800], Y[:1800], steps=4000, lr=3e-3)
    assert hist[-1][1] < 1e-2
    t0 = inputs.OPT_BASE.copy()
    solver.solves = 0
    exact = sg.newton_exact(solver, t0, tol=1e-6)
    t_star = exact[-1][0]
    n_exact = next(s for (t, hz, s) in exact if abs(t - t_star) < 1e-3)
    solver.solves = 0
    sur = sg.newton_surrogate(solver, net, t0, tol=1e-6)
    n_sur = next(s for (t, hz, s, kind) in sur if abs(t - t_star) < 1e-3)
    assert abs(sur[-1][0] - t_star) < 1e-3
    assert n_sur < n_exact, (n_sur, n_exact)
