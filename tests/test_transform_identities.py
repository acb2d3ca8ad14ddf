"""Identities the GPU kernels rely on, checked on the CPU with numpy (the kernels
themselves are covered by the GPU parity tests).

- A sequence zero-padded from n <= 512 to 1024 points: X[2k] = DFT_512(x)[k],
  X[2k+1] = DFT_512(x W_1024^n)[k]; the inverse at n < 512 (the crop) is
  IDFT_512(Y_even) + W_1024^-n IDFT_512(Y_odd) (unnormalised transforms).
- Rounding a float32 to TF32 (10 explicit mantissa bits), to nearest with ties
  away from zero, by adding half a unit of the last kept bit to the magnitude
  bits and clearing the 13 dropped bits; and the 3-pass split a_hi s_hi +
  a_hi s_lo + a_lo s_hi with the lo part passed unrounded and read by the
  tensor core from its upper 19 bits.
"""
import numpy as np


def _dft(x):
    return np.fft.fft(x)


def _idft_unnormalised(y):
    return np.fft.ifft(y) * len(y)


def test_zero_padded_1024_transform_as_two_512_point_transforms():
    rng = np.random.default_rng(5)
    for n in (257, 300, 511, 512):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        xp = np.zeros(1024, complex)
        xp[:n] = x
        X = _dft(xp)
        x512 = xp[:512]
        w = np.exp(-2j * np.pi * np.arange(512) / 1024)
        assert np.allclose(X[0::2], _dft(x512), atol=1e-9 * np.abs(X).max())
        assert np.allclose(X[1::2], _dft(x512 * w), atol=1e-9 * np.abs(X).max())


def test_cropped_1024_inverse_as_two_512_point_inverses():
    rng = np.random.default_rng(6)
    Y = rng.standard_normal(1024) + 1j * rng.standard_normal(1024)
    y = _idft_unnormalised(Y)[:512]
    w_inv = np.exp(2j * np.pi * np.arange(512) / 1024)
    z = _idft_unnormalised(Y[0::2]) + w_inv * _idft_unnormalised(Y[1::2])
    assert np.allclose(y, z, atol=1e-9 * np.abs(y).max())


def _tf32_round(v):
    bits = np.asarray(v, np.float32).view(np.uint32)
    return ((bits + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def _tf32_nearest_ties_away(v):
    """Reference: the nearest value with 10 explicit mantissa bits, ties away
    from zero, from the float64 value (finite normal inputs)."""
    v = np.asarray(v, np.float64)
    m, e = np.frexp(np.abs(v))                 # |v| = m 2^e, m in [0.5, 1)
    q = np.floor(m * 2048.0 + 0.5) / 2048.0    # 11 significant bits: 1 implicit + 10
    return (np.sign(v) * np.ldexp(q, e)).astype(np.float32)


def test_tf32_rounding_is_nearest_ties_away():
    rng = np.random.default_rng(7)
    v = (rng.standard_normal(200000) * np.exp(rng.uniform(-20, 20, 200000))).astype(np.float32)
    # exact ties: 10 kept bits then a single 1 in the first dropped position
    ties = (np.float32(1.0) + np.float32(2.0 ** -11) * (2 * rng.integers(0, 1024, 1000) + 1)).astype(np.float32)
    for x in (v, ties, -ties):
        assert np.array_equal(_tf32_round(x), _tf32_nearest_ties_away(x))


def _tf32_read(v):
    """What a TF32 operand contributes: the upper 19 bits (truncation)."""
    return (np.asarray(v, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def test_three_pass_split_product_error():
    rng = np.random.default_rng(8)
    a = rng.standard_normal(100000).astype(np.float32)
    s = rng.standard_normal(100000).astype(np.float32)
    a_hi, s_hi = _tf32_round(a), _tf32_round(s)
    a_lo = (a - a_hi).astype(np.float32)       # exact in float32
    s_lo = (s - s_hi).astype(np.float32)
    assert np.array_equal(a_hi.astype(np.float64) + a_lo, a.astype(np.float64))
    prod = (a_hi.astype(np.float64) * s_hi + a_hi.astype(np.float64) * _tf32_read(s_lo)
            + _tf32_read(a_lo).astype(np.float64) * s_hi)
    exact = a.astype(np.float64) * s.astype(np.float64)
    # dropped a_lo s_lo (<= 2^-22) and the truncated lo parts (<= 2^-21 each)
    assert np.max(np.abs(prod - exact) / np.abs(exact)) < 2.0 ** -19
