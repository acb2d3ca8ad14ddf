"""Pins of the oracle network (CPU): its backward pass against central
differences of its own forward pass, and the host bfloat16 rounding against
torch's conversion."""
import numpy as np
import torch

from oracle import mlp as omlp
from paper_1910_07054_gb300 import inputs


def test_oracle_backward_matches_finite_differences():
    I, H, O = 5, 7, 2
    rng = np.random.default_rng(3)
    w = inputs.mlp_init(I, H, O, seed=4).astype(np.float64)
    x = rng.standard_normal((6, I))
    gy = rng.standard_normal((6, O))
    gw, gx = omlp.backward(w, x, gy, I, H, O)

    def loss(wv, xv):
        return float(np.sum(omlp.forward(wv, xv, I, H, O)[0] * gy))

    h = 1e-6
    for k in rng.choice(w.size, 25, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        assert abs((loss(wp, x) - loss(wm, x)) / (2 * h) - gw[k]) < 1e-7 * max(1.0, abs(gw[k]))
    for s, i in [(0, 0), (3, 4), (5, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[s, i] += h
        xm[s, i] -= h
        assert abs((loss(w, xp) - loss(w, xm)) / (2 * h) - gx[s, i]) < 1e-7


def test_linear_limit():
    """With all hidden pre-activations tiny, tanh is the identity to first
    order and the network is the product of its weight matrices."""
    I, H, O = 3, 4, 2
    w = inputs.mlp_init(I, H, O, seed=1).astype(np.float64) * 1e-3
    W1, b1, W2, b2, W3, b3, W4, b4 = omlp.unpack(w, I, H, O)
    x = np.array([[0.2, -0.1, 0.3]])
    y, _ = omlp.forward(w, x, I, H, O)
    lin = ((x @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    assert np.allclose(y, lin @ W4.T + b4, rtol=1e-4, atol=1e-15)


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(0).standard_normal(5000).astype(np.float32) * 10
    x[:4] = [1.00390625, 1.01171875, -3.0, 0.0]
    vals, bits = inputs.bf16_round(x)
    ref = torch.tensor(x).to(torch.bfloat16)
    assert np.array_equal(bits.view(np.int16), ref.view(torch.int16).numpy())
    assert np.array_equal(vals, ref.float().numpy())
