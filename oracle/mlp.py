"""Oracle of the surrogate network (test infrastructure only).

Plain float64 numpy restatement of the multilayer perceptron the library runs
for the thickness optimisation of Sec. 4: I inputs, three tanh hidden layers of
H units, O linear outputs; parameter vector W1 [H][I], b1, W2 [H][H], b2,
W3 [H][H], b3, W4 [O][H], b4 (row-major W[out][in]).
"""
import numpy as np


def unpack(w, I, H, O):
    w = np.asarray(w, dtype=np.float64)
    shapes = [(H, I), (H,), (H, H), (H,), (H, H), (H,), (O, H), (O,)]
    out, k = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        out.append(w[k:k + n].reshape(sh))
        k += n
    assert k == w.size
    return out


def forward(w, x, I, H, O):
    """y [N, O] and the activations (x, h1, h2, h3)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(w, I, H, O)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    h3 = np.tanh(h2 @ W3.T + b3)
    return h3 @ W4.T + b4, (x, h1, h2, h3)


def backward(w, x, gy, I, H, O):
    """dLoss/dw (flat, same layout) and dLoss/dx for upstream gy = dLoss/dy."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(w, I, H, O)
    _, (x, h1, h2, h3) = forward(w, x, I, H, O)
    gy = np.asarray(gy, dtype=np.float64)
    d3 = (gy @ W4) * (1 - h3 ** 2)
    d2 = (d3 @ W3) * (1 - h2 ** 2)
    d1 = (d2 @ W2) * (1 - h1 ** 2)
    grads = [d1.T @ x, d1.sum(0), d2.T @ h1, d2.sum(0), d3.T @ h2, d3.sum(0), gy.T @ h3, gy.sum(0)]
    return np.concatenate([g.ravel() for g in grads]), d1 @ W1
