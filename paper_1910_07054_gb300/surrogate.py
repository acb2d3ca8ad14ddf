"""Surrogate-assisted thickness optimisation (Sec. 4 of the paper).

The paper drives one layer thickness of an MRAM stack by Newton iteration until
the mean z-field the pinned layers produce in the free layer vanishes.  Here a
small network, trained on samples the hybrid solver generates, maps the layer
thicknesses to that mean field and proposes the Newton steps; every proposal is
evaluated by the exact solver, which accepts it only if it reduces the residual
(otherwise an exact Newton step with the adjoint thickness derivative is taken).

The network runs in libdemag's kernels (demag_mlp_*); this module routes
tensors, normalises inputs and counts exact solves.
"""
import numpy as np
import torch

from . import _lib
from . import inputs


class ExactSolver:
    """Mean free-layer field of the optimisation stack for given thicknesses,
    counting every exact evaluation (a plan build plus an apply)."""

    def __init__(self, n, dx, Ms=inputs.MS_DEFAULT, precision=_lib.PREC_FP32):
        self.n, self.dx, self.Ms, self.precision = n, dx, Ms, precision
        dtype = torch.float64 if precision == _lib.PREC_FP64 else torch.float32
        self.m = torch.tensor(inputs.opt_stack_magnetization(n)[None], dtype=dtype, device="cuda")
        self.mean = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
        self.solves = 0

    def _plan(self, t):
        return _lib.Plan(self.n, self.n, self.dx, self.dx, [float(v) for v in t], precision=self.precision)

    def field(self, t):
        """Mean (Hx, Hy, Hz) / Ms over the free layer."""
        plan = self._plan(t)
        H = plan.apply(self.m, self.Ms)
        _lib.demag_layer_mean(H, self.precision, inputs.FREE_LAYER, self.mean)
        out = self.mean[0].cpu().numpy() / self.Ms
        plan.close()
        self.solves += 1
        return out

    def hz_and_slope(self, t, layer=inputs.OPT_LAYER):
        """Mean H_z / Ms of the free layer and its exact derivative in t[layer]
        (adjoint thickness derivative: two exact evaluations)."""
        plan = self._plan(t)
        H = plan.apply(self.m, self.Ms)
        _lib.demag_layer_mean(H, self.precision, inputs.FREE_LAYER, self.mean)
        hz = float(self.mean[0, 2].item()) / self.Ms
        gH = torch.zeros_like(self.m)
        gH[0, inputs.FREE_LAYER, 2] = 1.0 / (self.n * self.n * self.Ms)
        slope = _lib.demag_thickness_grad(plan.handle, self.m, gH, self.Ms, layer, info=plan.info)
        plan.close()
        self.solves += 2
        return hz, slope


def generate_samples(solver, thicknesses):
    """(thicknesses [N, L], mean free-layer field / Ms [N, 3]) from the solver."""
    Y = np.stack([solver.field(t) for t in thicknesses])
    return np.asarray(thicknesses, dtype=np.float64), Y


def save_samples(path, T, Y):
    """Cache a training set (one exact solve per row) in an .npz file."""
    np.savez(path, T=np.asarray(T, dtype=np.float64), Y=np.asarray(Y, dtype=np.float64))


def load_samples(path):
    """(T, Y) from save_samples."""
    with np.load(path) as f:
        return f["T"].copy(), f["Y"].copy()


class Surrogate:
    """I -> H -> H -> H -> O tanh network in bf16 weights / float sums."""

    def __init__(self, I=8, H=64, O=3, seed=0, device="cuda"):
        self.I, self.H, self.O = I, H, O
        self.device = device
        self.P = _lib.demag_mlp_param_count(I, H, O)
        self._set_weights(inputs.mlp_init(I, H, O, seed))
        self.m1 = torch.zeros_like(self.w)
        self.m2 = torch.zeros_like(self.w)
        self.step = 0
        self.x_mean = np.zeros(I)
        self.x_std = np.ones(I)
        self.y_scale = np.ones(O)

    def _set_weights(self, w0):
        # float master weights, their bf16 copy (what the kernels read) and the gradient
        w0 = np.asarray(w0, dtype=np.float32)
        self.w = torch.tensor(w0, device=self.device)
        _, bits = inputs.bf16_round(w0)
        self.wb = torch.from_numpy(bits.view(np.int16)).to(self.device).view(torch.bfloat16)
        self.g = torch.zeros_like(self.w)

    def state(self):
        """Everything training needs to resume: master weights, Adam moments and
        step, and the input / output normalisation (numpy arrays)."""
        return {"shape": np.array([self.I, self.H, self.O]), "w": self.w.cpu().numpy(),
                "m1": self.m1.cpu().numpy(), "m2": self.m2.cpu().numpy(), "step": np.array(self.step),
                "x_mean": np.asarray(self.x_mean), "x_std": np.asarray(self.x_std),
                "y_scale": np.asarray(self.y_scale)}

    def save(self, path):
        """Checkpoint the network (state()) to an .npz file."""
        np.savez(path, **self.state())

    @classmethod
    def load(cls, path, device="cuda"):
        """A network restored from save(): fit() continues its Adam run."""
        with np.load(path) as f:
            st = {k: f[k].copy() for k in f.files}
        I, H, O = (int(v) for v in st["shape"])
        net = cls(I, H, O, device=device)
        if st["w"].shape != (net.P,):
            raise ValueError("checkpoint holds %d parameters, an %d-%d-%d network has %d"
                             % (st["w"].size, I, H, O, net.P))
        net._set_weights(st["w"])
        net.m1 = torch.tensor(st["m1"], device=device)
        net.m2 = torch.tensor(st["m2"], device=device)
        net.step = int(st["step"])
        net.x_mean, net.x_std, net.y_scale = st["x_mean"], st["x_std"], st["y_scale"]
        return net

    def _x(self, t):
        x = (np.atleast_2d(t) - self.x_mean) / self.x_std
        return torch.tensor(x, dtype=torch.float32, device=self.device).contiguous()

    def fit(self, T, Y, steps=3000, lr=3e-3, log_every=0):
        """Full-batch Adam on the mean squared error of the scaled outputs."""
        T, Y = np.asarray(T), np.asarray(Y)
        self.x_mean, self.x_std = T.mean(0), T.std(0) + 1e-12
        self.y_scale = np.abs(Y).max(0) + 1e-30
        x = self._x(T)
        yt = torch.tensor(Y / self.y_scale, dtype=torch.float32, device=self.device).contiguous()
        y = torch.empty_like(yt)
        gy = torch.empty_like(yt)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        history = []
        for k in range(steps):
            loss.zero_()
            _lib.demag_mlp_forward(self.wb, x, y, self.I, self.H, self.O)
            _lib.demag_mlp_mse(y, yt, gy, loss)
            _lib.demag_mlp_backward(self.wb, x, gy, self.g, None, self.I, self.H, self.O)
            self.step += 1
            _lib.demag_mlp_adam(self.w, self.wb, self.g, self.m1, self.m2, lr, 0.9, 0.999, 1e-8, self.step)
            if log_every and (k % log_every == 0 or k == steps - 1):
                history.append((k, float(loss.item())))
        if not history:
            history.append((steps - 1, float(loss.item())))
        return history

    def predict(self, t):
        x = self._x(t)
        y = torch.empty(x.shape[0], self.O, dtype=torch.float32, device=self.device)
        _lib.demag_mlp_forward(self.wb, x, y, self.I, self.H, self.O)
        return y.double().cpu().numpy() * self.y_scale

    def slope(self, t, out=2, layer=inputs.OPT_LAYER):
        """d(output `out`)/d t[layer] through the network (its input gradient)."""
        x = self._x(t)
        gy = torch.zeros(x.shape[0], self.O, dtype=torch.float32, device=self.device)
        gy[:, out] = 1.0
        gx = torch.empty_like(x)
        _lib.demag_mlp_backward(self.wb, x, gy, None, gx, self.I, self.H, self.O)
        return gx[:, layer].double().cpu().numpy() * self.y_scale[out] / self.x_std[layer]


def newton_exact(solver, t0, tol=1e-5, max_iter=20, layer=inputs.OPT_LAYER, bounds=(0.3, 6.0)):
    """Newton on t[layer] with the exact adjoint derivative.  Returns the
    history [(t_layer, hz, exact solves so far)]."""
    t = np.array(t0, dtype=np.float64)
    hist = []
    for _ in range(max_iter):
        hz, d = solver.hz_and_slope(t, layer)
        hist.append((t[layer], hz, solver.solves))
        step = -hz / d
        t[layer] = float(np.clip(t[layer] + step, *bounds))
        if abs(step) < tol:
            break
    return hist


def newton_surrogate(solver, net, t0, tol=1e-5, max_iter=20, layer=inputs.OPT_LAYER,
                     bounds=(0.3, 6.0)):
    """Surrogate-proposed steps judged by the exact solver.

    Each proposal is the root in t[layer] of the network's H_z corrected to the
    exact evaluations along the path: m(x) = hz_k + s (net(x) - net(t_k)), with
    hz_k the last accepted exact value at t_k (the network supplies the shape,
    the solver the level) and, once two exact points are known, s the ratio of
    their exact to their network difference (the solver also fixes the scale;
    s = 1 before that, clipped to [1/4, 4]).  The solver evaluates the proposal;
    it is accepted if |H_z| drops, otherwise an exact Newton step with the
    adjoint derivative is taken.
    Returns the history [(t_layer, hz, exact solves so far, 'accept' | 'exact')].
    """
    t = np.array(t0, dtype=np.float64)
    hz = solver.field(t)[2]
    hist = [(t[layer], hz, solver.solves, "start")]
    prev = None  # (network value, exact value) at the previous exact point
    for _ in range(max_iter):
        n_t = net.predict(t)[0, 2]
        scale = 1.0
        if prev is not None and abs(n_t - prev[0]) > 1e-12:
            scale = float(np.clip((hz - prev[1]) / (n_t - prev[0]), 0.25, 4.0))
        tp = t.copy()
        for _ in range(30):  # Newton on the corrected surrogate alone: no exact solves
            r = scale * (net.predict(tp)[0, 2] - n_t) + hz
            d = scale * net.slope(tp, 2, layer)[0]
            if d == 0.0:
                break
            dt = -r / d
            tp[layer] = float(np.clip(tp[layer] + dt, *bounds))
            if abs(dt) < 1e-9:
                break
        step = tp[layer] - t[layer]
        hz_p = solver.field(tp)[2]
        if abs(hz_p) < abs(hz):
            prev = (n_t, hz)
            t, hz = tp, hz_p
            hist.append((t[layer], hz, solver.solves, "accept"))
        else:
            hz0, d = solver.hz_and_slope(t, layer)
            prev = (n_t, hz)
            t = t.copy()
            step = -hz0 / d
            t[layer] = float(np.clip(t[layer] + step, *bounds))
            hz = solver.field(t)[2]
            hist.append((t[layer], hz, solver.solves, "exact"))
        if abs(step) < tol:
            break
    return hist
