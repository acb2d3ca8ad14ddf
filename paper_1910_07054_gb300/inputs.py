"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds no arithmetic of the demagnetization method: only layer
stacks, sizes and seeded magnetization patterns shaped like the paper's
multilayers (Sec. 3.2 scaling runs at 256 x 256 cells, the SAFM stack of Sec. 4).
All magnetization arrays are float64 [B, L, 3, ny, nx] or [L, 3, ny, nx],
x fastest, unit vectors (or zero in non-magnetic cells).
"""
import numpy as np

MS_DEFAULT = 8.0e5  # A/m

# Named workloads: grid, cell size (nm) and layer thicknesses (nm).
CONFIGS = {
    # 32 x 32 x 3, random unit vectors, float64 path, checked by direct summation
    "plain32": dict(nx=32, ny=32, dx=2.0, dy=2.0, thickness=[1.0, 0.5, 2.0], batch=1),
    # MRAM-like stack, 256 x 256 x 8
    "mram256": dict(nx=256, ny=256, dx=2.0, dy=2.0,
                    thickness=[1.0, 0.8, 1.2, 0.9, 5.0, 1.5, 0.7, 2.0], batch=1),
    # layer scaling + batch: 512 x 512 x 64, 16 states
    "scale512": dict(nx=512, ny=512, dx=2.0, dy=2.0, thickness=None, batch=16,
                     thickness_range=(0.5, 3.0), L=64, seed=0),
    # differentiation: 256 x 256 x 10
    "grad256": dict(nx=256, ny=256, dx=2.0, dy=2.0, thickness=None, batch=1,
                    thickness_range=(0.7, 4.0), L=10, seed=0),
}


def thicknesses(name):
    """Layer thicknesses (nm) of a named workload; seeded uniform draws where ranged."""
    c = CONFIGS[name]
    if c["thickness"] is not None:
        return np.asarray(c["thickness"], dtype=np.float64)
    lo, hi = c["thickness_range"]
    rng = np.random.default_rng(c["seed"])
    return rng.uniform(lo, hi, size=c["L"])


def random_unit_vectors(shape, seed):
    """Unit vectors uniform on the sphere: normalised N(0,1) triples.

    shape is the leading shape; the result has shape (*shape[:-2], 3, *shape[-2:])
    when shape = (..., ny, nx), i.e. a vector axis is inserted before y.
    """
    rng = np.random.default_rng(seed)
    lead, (ny, nx) = tuple(shape[:-2]), tuple(shape[-2:])
    v = rng.standard_normal(lead + (3, ny, nx))
    v /= np.linalg.norm(v, axis=-3, keepdims=True)
    return v


def mram_magnetization(nx, ny, L, seed=0, batch=None):
    """Mixed pattern for the MRAM-like stack: odd layers (1-based) carry two
    half-plane domains, m = +z for x < nx/2 and -z beyond; even layers carry
    seeded random unit vectors."""
    B = 1 if batch is None else batch
    m = np.zeros((B, L, 3, ny, nx))
    rnd = random_unit_vectors((B, L, ny, nx), seed)
    for l in range(L):
        if l % 2 == 0:  # layers 1, 3, 5, ... (1-based)
            m[:, l, 2, :, : nx // 2] = 1.0
            m[:, l, 2, :, nx // 2:] = -1.0
        else:
            m[:, l] = rnd[:, l]
    return m[0] if batch is None else m


def disk_mask(nx, ny):
    """Cells whose centre lies inside the disk inscribed in the grid."""
    yc = (np.arange(ny) + 0.5) - ny / 2
    xc = (np.arange(nx) + 0.5) - nx / 2
    r2 = (xc[None, :] / (nx / 2)) ** 2 + (yc[:, None] / (ny / 2)) ** 2
    return r2 <= 1.0


def safm_stack(t_middle, n=64, diameter=60.0):
    """Sec. 4 SAFM stack: layers [5, 1, t, 1, 3] nm on an n x n grid spanning the
    60 nm diameter; m = +z in layer 1 and -z in layer 3 inside the disk, zero in
    the spacers (layers 2, 4) and in the free layer (layer 5), whose field is
    the objective.  Returns (dx, thickness, m[5, 3, n, n])."""
    dx = diameter / n
    th = np.array([5.0, 1.0, float(t_middle), 1.0, 3.0])
    mask = disk_mask(n, n)
    m = np.zeros((5, 3, n, n))
    m[0, 2][mask] = 1.0
    m[2, 2][mask] = -1.0
    return dx, th, m


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest, ties to even).  Returns the
    rounded values as float32 and their 16-bit patterns (uint16)."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16).astype(np.uint16)
    back = (rounded.astype(np.uint32) << 16).view(np.float32)
    return back, rounded


def mlp_init(I, H, O, seed):
    """Seeded initial parameters (uniform, fan-in scaled), flat float32 vector."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((H, I), (H, H), (H, H), (O, H)):
        lim = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(rng.uniform(-lim, lim, size=fan_out))
    return np.concatenate(parts).astype(np.float32)


# Sec. 4-like optimisation stack on the MRAM-like thicknesses (1-based layers):
# layers 1, 3 pinned +z and layer 5 pinned -z inside the disk inscribed in
# the grid; layers 2, 4, 6, 7 spacers; layer 8 the free layer (m = 0), whose
# mean z-field is the objective; layer 5's thickness is the design variable.
OPT_BASE = np.array([1.0, 0.8, 1.2, 0.9, 5.0, 1.5, 0.7, 2.0])
OPT_LAYER = 4   # 0-based index of layer 5
FREE_LAYER = 7  # 0-based index of layer 8


def opt_stack_magnetization(n):
    mask = disk_mask(n, n)
    m = np.zeros((len(OPT_BASE), 3, n, n))
    m[0, 2][mask] = 1.0
    m[2, 2][mask] = 1.0
    m[4, 2][mask] = -1.0
    return m


def opt_samples(count, seed, t5_range=(0.5, 5.0), jitter=0.10):
    """Thickness sets: layer 5 uniform in t5_range, the others the base values
    jittered uniformly by +-jitter (relative)."""
    rng = np.random.default_rng(seed)
    t = OPT_BASE[None, :] * (1.0 + rng.uniform(-jitter, jitter, size=(count, len(OPT_BASE))))
    t[:, OPT_LAYER] = rng.uniform(t5_range[0], t5_range[1], size=count)
    return t
