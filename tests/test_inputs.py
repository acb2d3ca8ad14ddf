"""The seeded input recipe (paper_1910_07054_gb300/inputs.py): determinism,
shapes, unit vectors, the MRAM-like domain pattern, ranged thickness draws, the
SAFM and optimisation stacks, and the bfloat16 rounding used for the surrogate's
weights."""
import numpy as np

from paper_1910_07054_gb300 import inputs


def test_random_unit_vectors_seeded_and_normalised():
    a = inputs.random_unit_vectors((2, 3, 5, 7), seed=11)
    b = inputs.random_unit_vectors((2, 3, 5, 7), seed=11)
    c = inputs.random_unit_vectors((2, 3, 5, 7), seed=12)
    assert a.shape == (2, 3, 3, 5, 7)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.allclose(np.linalg.norm(a, axis=-3), 1.0, atol=1e-14)
    # uniform on the sphere: each component has mean 0 and variance 1/3
    v = inputs.random_unit_vectors((64, 64), seed=0).reshape(3, -1)
    assert np.all(np.abs(v.mean(axis=1)) < 0.03)
    assert np.all(np.abs(v.var(axis=1) - 1 / 3) < 0.02)


def test_mram_pattern():
    nx, ny, L = 10, 6, 5
    m = inputs.mram_magnetization(nx, ny, L, seed=3)
    assert m.shape == (L, 3, ny, nx)
    for l in range(0, L, 2):  # layers 1, 3, 5 (1-based): two half-plane z domains
        assert np.all(m[l, :2] == 0.0)
        assert np.all(m[l, 2, :, : nx // 2] == 1.0) and np.all(m[l, 2, :, nx // 2:] == -1.0)
    for l in range(1, L, 2):  # even layers: random unit vectors
        assert np.allclose(np.linalg.norm(m[l], axis=0), 1.0)
    mb = inputs.mram_magnetization(nx, ny, L, seed=3, batch=2)
    assert mb.shape == (2, L, 3, ny, nx) and np.array_equal(mb[0], m)


def test_named_thicknesses():
    assert np.array_equal(inputs.thicknesses("mram256"), [1.0, 0.8, 1.2, 0.9, 5.0, 1.5, 0.7, 2.0])
    t = inputs.thicknesses("scale512")
    assert t.shape == (64,) and np.all((t >= 0.5) & (t < 3.0))
    assert np.array_equal(t, inputs.thicknesses("scale512"))  # seeded
    g = inputs.thicknesses("grad256")
    assert g.shape == (10,) and np.all((g >= 0.7) & (g < 4.0))


def test_safm_and_optimisation_stacks():
    dx, th, m = inputs.safm_stack(1.3, n=32)
    assert dx == 60.0 / 32 and np.array_equal(th, [5.0, 1.0, 1.3, 1.0, 3.0])
    mask = inputs.disk_mask(32, 32)
    assert np.all(m[0, 2][mask] == 1.0) and np.all(m[2, 2][mask] == -1.0)
    assert np.all(m[0, 2][~mask] == 0.0)
    assert np.all(m[[1, 3, 4]] == 0.0)  # spacers and the free layer carry no moment
    # the inscribed disk covers about pi/4 of the square grid
    assert abs(mask.mean() - np.pi / 4) < 0.02
    mo = inputs.opt_stack_magnetization(16)
    assert np.all(mo[inputs.FREE_LAYER] == 0.0)
    T = inputs.opt_samples(500, seed=1)
    base = inputs.OPT_BASE
    others = np.delete(np.arange(len(base)), inputs.OPT_LAYER)
    assert np.all(np.abs(T[:, others] / base[others] - 1.0) <= 0.10 + 1e-12)
    assert np.all((T[:, inputs.OPT_LAYER] >= 0.5) & (T[:, inputs.OPT_LAYER] < 5.0))


def test_bf16_round_nearest_ties_to_even():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 3.0e-3], np.float32)
    back, bits = inputs.bf16_round(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1); 1 + 3 2^-8 ties up to 1 + 2^-6
    assert back[0] == 1.0 and back[1] == 1.0 and back[2] == np.float32(1.0 + 2.0 ** -6)
    assert back[3] == 1.0  # below half a unit
    assert back[4] == -2.5  # exactly representable
    assert abs(back[5] - 3.0e-3) <= 2.0 ** -8 * 3.0e-3
    assert np.array_equal((bits.astype(np.uint32) << 16).view(np.float32), back)
