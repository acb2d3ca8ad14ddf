"""Checkpoint and resume of the surrogate (host side, no GPU): a network's state
(master weights, Adam moments and step, normalisation) and a cached training
set survive an .npz round trip unchanged, the restored bf16 weights are the
nearest-even rounding of the master weights (what the Adam kernel keeps), and a
checkpoint of another network shape is refused."""
import numpy as np
import pytest
import torch

from paper_1910_07054_gb300 import surrogate as sg


def _trained_like(seed):
    net = sg.Surrogate(I=8, H=16, O=3, seed=seed, device="cpu")
    rng = np.random.default_rng(seed)
    net._set_weights(rng.standard_normal(net.P).astype(np.float32))
    net.m1 = torch.tensor(rng.standard_normal(net.P).astype(np.float32))
    net.m2 = torch.tensor(rng.random(net.P).astype(np.float32))
    net.step = 1234
    net.x_mean = rng.standard_normal(8)
    net.x_std = rng.random(8) + 0.5
    net.y_scale = rng.random(3) + 1e-3
    return net


def test_network_state_round_trip(tmp_path):
    net = _trained_like(5)
    path = tmp_path / "net.npz"
    net.save(path)
    back = sg.Surrogate.load(path, device="cpu")
    a, b = net.state(), back.state()
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert back.step == 1234 and (back.I, back.H, back.O) == (8, 16, 3)
    assert torch.equal(back.wb, back.w.to(torch.bfloat16))
    assert torch.equal(back.wb, net.wb)


def test_checkpoint_of_another_shape_is_refused(tmp_path):
    net = _trained_like(6)
    st = net.state()
    st["w"] = st["w"][:-1]
    path = tmp_path / "bad.npz"
    np.savez(path, **st)
    with pytest.raises(ValueError):
        sg.Surrogate.load(path, device="cpu")


def test_training_set_round_trip(tmp_path):
    rng = np.random.default_rng(7)
    T, Y = rng.random((50, 8)), rng.standard_normal((50, 3))
    path = tmp_path / "samples.npz"
    sg.save_samples(path, T, Y)
    T2, Y2 = sg.load_samples(path)
    assert np.array_equal(T, T2) and np.array_equal(Y, Y2)
