"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Tolerances: float64 plans within 1e-11 relative L2 of the oracle field, float32
plans within 1e-5 relative L2 (the accuracy target of this library); the
tensor evaluation within 5e-13 of the largest component of the exact
_Float128 tensor.
"""
import numpy as np
import pytest
import torch

import paper_1910_07054_gb300 as dm
from oracle import demag as odm
from oracle import newell as onw
from paper_1910_07054_gb300 import inputs
from _cases import quad_kernels, reading_kernels, rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _gpu_field(nx, ny, dx, dy, th, m, Ms, prec, max_batch=None):
    dtype = torch.float64 if prec == dm.PREC_FP64 else torch.float32
    mt = torch.as_tensor(m, dtype=dtype, device="cuda").contiguous()
    B = mt.shape[0] if mt.dim() == 5 else 1
    plan = dm.Plan(nx, ny, dx, dy, th, precision=prec, max_batch=max_batch or B)
    H = plan.apply(mt, Ms)
    torch.cuda.synchronize()
    out = H.double().cpu().numpy()
    plan.close()
    return out


def _random_geometries(n, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for k in range(n):
        ti, tj = rng.uniform(0.3, 5.0, size=2)
        if k % 4 == 3:  # fully unequal cuboids
            t = rng.uniform(0.5, 3.0, size=3)
            s = rng.uniform(0.5, 3.0, size=3)
        else:
            t = np.array([2.0, 2.0, ti])
            s = np.array([2.0, 2.0, tj])
        R = float(np.exp(rng.uniform(np.log(0.3), np.log(800.0))))
        d = rng.standard_normal(3)
        d[2] *= rng.uniform(0.01, 1.0)
        d *= R / np.linalg.norm(d)
        X, Y, Z = round(d[0] / 2) * 2.0, round(d[1] / 2) * 2.0, float(d[2])
        rows.append([X, Y, Z, *t, *s])
    rows += [[0, 0, 0, 1, 1, 1, 1, 1, 1], [0, 0, 0, 2, 2, 0.5, 2, 2, 0.5], [2, 0, 0, 2, 2, 1, 2, 2, 1],
             [0, 0, 1.0, 2, 2, 1.0, 2, 2, 0.5], [0, 0, -2.0, 2, 2, 1.0, 2, 2, 2.0]]
    return np.array(rows, dtype=np.float64)


def test_tensor_points_match_oracle():
    g = _random_geometries(300, seed=11)
    gt = torch.tensor(g, device="cuda")
    out = torch.empty(len(g), 6, dtype=torch.float64, device="cuda")
    dm.demag_tensor_points(gt, out)
    torch.cuda.synchronize()
    N = out.cpu().numpy()
    worst_q = worst_r = 0.0
    for k, row in enumerate(g):
        X, Y, Z = row[:3]
        nq = onw.tensor(X, Y, Z, row[3:6], row[6:9], mode=onw.EXACT_Q)
        nr = onw.tensor(X, Y, Z, row[3:6], row[6:9], mode=onw.READING_D)
        sc = np.abs(nq).max()
        worst_q = max(worst_q, np.abs(N[k] - nq).max() / sc)
        worst_r = max(worst_r, np.abs(N[k] - nr).max() / sc)
    assert worst_q < 5e-13, worst_q
    assert worst_r < 5e-13, worst_r
    # self term of a cube
    assert np.allclose(N[len(g) - 5, :3], 1.0 / 3.0, atol=1e-15)


def _stored_ky(Py, path=1):
    """y-frequency held by each stored entry u (the documented order of
    demag_plan_tensor: bit-reversed positions, one partner of each mirror pair;
    natural order on the 512-point path 5)."""
    if path == 5:
        return np.arange(Py // 2 + 1)
    n = Py.bit_length() - 1
    out = []
    for u in range(Py // 2 + 1):
        if u < 2:
            p1 = u
        else:
            m = (u - 1).bit_length()
            p1 = (1 << m) + u - (1 << (m - 1)) - 1
        k = int(format(p1, "0%db" % n)[::-1], 2)
        out.append(min(k, Py - k))
    return np.array(out)


@pytest.mark.parametrize("nx,ny,th", [(7, 5, (1.0, 0.5, 2.0)), (4, 9, (0.8,)), (12, 3, (0.6, 3.0)),
                                      (16, 16, (1.0, 2.0)), (200, 140, (1.0, 2.0))])
def test_plan_tensor_matches_oracle_spectrum(nx, ny, th):
    """The stored Fourier tensor equals the oracle's kernels placed on the same
    padded grid and transformed by numpy's FFT (quadrant, divided by Px Py),
    in the documented storage order."""
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_FP64)
    info = plan.info
    Px, Py, L, npairs, QyS = info["Px"], info["Py"], info["L"], info["npairs"], info["QyS"]
    Kx, Qy = Px // 2 + 1, Py // 2 + 1
    out = torch.empty(Kx * npairs * 6 * QyS, dtype=torch.float64, device="cuda")
    dm.demag_plan_tensor(plan.handle, out)
    torch.cuda.synchronize()
    T = out.cpu().numpy().reshape(Kx, npairs, 6, QyS)
    plan.close()
    assert np.all(T[..., Qy:] == 0.0)
    ky_of_u = _stored_ky(Py, info["path"])
    if nx == 200:
        assert info["path"] == 5
    assert sorted(ky_of_u.tolist()) == list(range(Qy))
    K = reading_kernels(nx, ny, 2.0, 2.0, tuple(th))
    pairs = [(i, j) for i in range(L) for j in range(i, L)]
    qs = np.arange(-(ny - 1), ny) % Py
    ps = np.arange(-(nx - 1), nx) % Px
    for P, (i, j) in enumerate(pairs):
        Kp = np.zeros((6, Py, Px))
        Kp[:, qs[:, None], ps[None, :]] = K[i, j]
        S = np.fft.fft2(Kp) / (Px * Py)
        ref = np.stack([S[0].real, S[1].real, S[2].real, S[3].real, S[4].imag, S[5].imag])
        # the structure: even components have real spectra, odd ones imaginary
        assert np.abs(S[:4].imag).max() < 1e-14 and np.abs(S[4:].real).max() < 1e-14
        ref_u = ref[:, ky_of_u, :Kx]                  # [component, u, kx]
        got_u = np.transpose(T[:, P, :, :Qy], (1, 2, 0))
        sc = np.abs(ref_u).max()
        assert np.abs(got_u - ref_u).max() < 1e-12 * sc


def test_plain32_fp64_matches_direct_sum():
    """32 x 32 x 3 layers of 1.0 / 0.5 / 2.0 nm, random unit vectors, float64:
    the GPU field against brute-force summation with the exact _Float128 tensor."""
    c = inputs.CONFIGS["plain32"]
    th = tuple(c["thickness"])
    m = inputs.random_unit_vectors((len(th), c["ny"], c["nx"]), seed=0)
    Ms = inputs.MS_DEFAULT
    K = quad_kernels(c["nx"], c["ny"], c["dx"], c["dy"], th)
    H_ref = odm.direct_sum(K, m, Ms)
    H = _gpu_field(c["nx"], c["ny"], c["dx"], c["dy"], th, m[None], Ms, dm.PREC_FP64)[0]
    assert rel_l2(H, H_ref) < TOL64


RAGGED = [(7, 5, (1.0, 0.5, 2.0)), (1, 1, (2.0,)), (33, 17, (0.9, 1.3, 0.4, 2.2)), (16, 1, (1.0, 1.0)),
          (3, 40, (0.7,)), (20, 20, (0.5, 1.5, 0.5, 2.5, 1.0, 0.8, 3.0, 1.1)),
          # 512-point transforms (radix-8 kernels), ragged rows and columns
          (200, 140, (1.0, 0.5, 2.0)), (129, 256, (0.8, 1.7)), (256, 131, (1.2,)),
          # 512-point columns under short rows, and 512-point rows over short columns
          (5, 200, (1.0, 0.6)), (200, 6, (0.9, 2.0)),
          # 1024-point rows (two 512-point transforms per row pair), ragged and full
          (300, 19, (1.0, 0.5, 2.0)), (512, 6, (1.3,))]


@pytest.mark.parametrize("nx,ny,th", RAGGED)
@pytest.mark.parametrize("prec", [dm.PREC_FP64, dm.PREC_FP32])
def test_ragged_grids_match_oracle_hybrid(nx, ny, th, prec):
    m = inputs.random_unit_vectors((len(th), ny, nx), seed=nx * 100 + ny)
    K = reading_kernels(nx, ny, 2.0, 1.5, th)
    H_ref = odm.hybrid(K, m, 1.0)
    H = _gpu_field(nx, ny, 2.0, 1.5, th, m[None], 1.0, prec)[0]
    assert rel_l2(H, H_ref) < (TOL64 if prec == dm.PREC_FP64 else TOL32)


@pytest.mark.parametrize("L", range(1, 12))
def test_streamed_columns_every_layer_count(L):
    """Float plans with 512-point columns and L <= 11 take the kernel that streams
    the tensor through shared memory (every unrolled pair count, ragged grid,
    batch of two states); no bounded wait may give up."""
    rng = np.random.default_rng(40 + L)
    th = tuple(np.round(rng.uniform(0.4, 3.0, L), 3))
    nx, ny = 150, 131
    m = inputs.random_unit_vectors((2, L, ny, nx), seed=L)
    K = reading_kernels(nx, ny, 2.0, 1.5, th)
    H = _gpu_field(nx, ny, 2.0, 1.5, th, m, 1.0, dm.PREC_FP32, max_batch=2)
    assert dm.demag_wait_timeouts() == 0
    for b in range(2):
        assert rel_l2(H[b], odm.hybrid(K, m[b], 1.0)) < TOL32


def test_sixteen_layers_fp32():
    th = tuple(np.round(np.linspace(0.5, 3.0, 16), 3))
    nx = ny = 24
    m = inputs.random_unit_vectors((16, ny, nx), seed=21)
    K = reading_kernels(nx, ny, 2.0, 2.0, th)
    H_ref = odm.hybrid(K, m, 1.0)
    H = _gpu_field(nx, ny, 2.0, 2.0, th, m[None], 1.0, dm.PREC_FP32)[0]
    assert rel_l2(H, H_ref) < TOL32


def test_mram256_fp32_full_size():
    """256 x 256 x 8 MRAM-like stack, float32 apply, the launch the bench times."""
    c = inputs.CONFIGS["mram256"]
    th = tuple(c["thickness"])
    m = inputs.mram_magnetization(c["nx"], c["ny"], len(th), seed=0)
    K = reading_kernels(c["nx"], c["ny"], c["dx"], c["dy"], th)
    H_ref = odm.hybrid(K, m, inputs.MS_DEFAULT)
    H = _gpu_field(c["nx"], c["ny"], c["dx"], c["dy"], th, m[None], inputs.MS_DEFAULT, dm.PREC_FP32)[0]
    assert rel_l2(H, H_ref) < TOL32


def test_batch_states_are_independent():
    nx, ny, th = 20, 12, (1.0, 0.6, 2.0)
    m = inputs.random_unit_vectors((3, len(th), ny, nx), seed=31)
    Hb = _gpu_field(nx, ny, 2.0, 2.0, th, m, 5.0, dm.PREC_FP32)
    for b in range(3):
        Hs = _gpu_field(nx, ny, 2.0, 2.0, th, m[b:b + 1], 5.0, dm.PREC_FP32, max_batch=3)[0]
        assert np.array_equal(Hb[b], Hs)


def test_host_entry_point_matches_device():
    nx, ny, th = 18, 10, (1.0, 0.6, 2.0)
    m = inputs.random_unit_vectors((2, len(th), ny, nx), seed=41)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_FP32, max_batch=2)
    mh = torch.tensor(m, dtype=torch.float32).pin_memory()
    Hh = torch.empty_like(mh).pin_memory()
    dm.demag_apply_host(plan.handle, mh, 3.0, Hh)          # pinned: kernels access host memory
    mp = torch.tensor(m, dtype=torch.float32)
    Hp = torch.empty_like(mp)
    dm.demag_apply_host(plan.handle, mp, 3.0, Hp)          # pageable: staged copies
    Hd = plan.apply(mh.cuda(), 3.0).cpu()
    plan.close()
    assert torch.equal(Hh, Hd)
    assert torch.equal(Hp, Hd)


def test_host_entry_point_512_point_path():
    """Pinned host buffers on the 512-point kernels (direct host access)."""
    nx, ny, th = 200, 140, (1.0, 0.5, 2.0)
    m = inputs.random_unit_vectors((1, len(th), ny, nx), seed=42)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_FP32)
    assert plan.info["path"] == 5
    mh = torch.tensor(m, dtype=torch.float32).pin_memory()
    Hh = torch.empty_like(mh).pin_memory()
    dm.demag_apply_host(plan.handle, mh, 3.0, Hh)
    Hd = plan.apply(mh.cuda(), 3.0).cpu()
    plan.close()
    assert torch.equal(Hh, Hd)


@pytest.mark.parametrize("nx,ny,th,prec,B", [
    (200, 140, (1.0, 0.5, 2.0), dm.PREC_FP32, 5),        # 512-point rows, fused 512-point columns
    (300, 20, (1.0, 0.5, 2.0, 0.8), dm.PREC_SPLIT_BF16, 3),  # 1024-point rows, split columns
    (20, 12, (1.0, 0.6), dm.PREC_FP64, 4),                # generic kernels, double
])
def test_host_entry_point_pipelined_batch(nx, ny, th, prec, B):
    """Pinned buffers and a batch: the chunked copies overlapped with the row
    transforms give the device field bit for bit, call after call; a pageable
    output buffer takes the plain staged copies."""
    dtype = torch.float64 if prec == dm.PREC_FP64 else torch.float32
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=prec, max_batch=B)
    for seed in (51, 52):
        m = inputs.random_unit_vectors((B, len(th), ny, nx), seed=seed)
        mh = torch.tensor(m, dtype=dtype).pin_memory()
        Hh = torch.full_like(mh, float("nan")).pin_memory()
        dm.demag_apply_host(plan.handle, mh, 3.0, Hh)
        Hd = plan.apply(mh.cuda(), 3.0).cpu()
        assert torch.equal(Hh, Hd)
        Hp = torch.empty_like(mh)  # pageable
        dm.demag_apply_host(plan.handle, mh, 3.0, Hp)
        assert torch.equal(Hp, Hd)
    plan.close()


def test_host_entry_point_async_stream_of_batches():
    """demag_apply_host_async: consecutive batches on alternating host buffers,
    one wait at the end, every field equal to the device apply bit for bit."""
    nx, ny, th, B = 300, 20, (1.0, 0.5, 2.0, 0.8), 3
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_SPLIT_BF16, max_batch=B)
    ms = [inputs.random_unit_vectors((B, len(th), ny, nx), seed=60 + k) for k in range(4)]
    mh = [torch.tensor(m, dtype=torch.float32).pin_memory() for m in ms]
    Hh = [torch.full_like(x, float("nan")).pin_memory() for x in mh]
    for k in range(4):
        dm.demag_apply_host_async(plan.handle, mh[k], 3.0, Hh[k])
    dm.demag_apply_host_wait(plan.handle)
    for k in range(4):
        assert torch.equal(Hh[k], plan.apply(mh[k].cuda(), 3.0).cpu()), k
    with pytest.raises(dm.DemagError):
        dm.demag_apply_host_async(plan.handle, torch.zeros_like(mh[0]), 3.0, Hh[0])  # pageable input
    plan.close()


def test_uniform_film_gpu():
    n, t, Ms = 63, 0.5, 8e5
    m = np.zeros((1, 1, 3, n, n))
    m[0, 0, 2] = 1.0
    H = _gpu_field(n, n, 2.0, 2.0, (t,), m, Ms, dm.PREC_FP64)[0, 0]
    c = n // 2
    film = onw.tensor(c * 2.0, c * 2.0, 0.0, (2.0, 2.0, t), (n * 2.0, n * 2.0, t))
    assert H[2, c, c] == pytest.approx(-Ms * film[2], rel=1e-11)


def test_gpu_argument_errors():
    plan = dm.Plan(8, 8, 2.0, 2.0, (1.0, 2.0), precision=dm.PREC_FP32, max_batch=1)
    m = torch.zeros(2, 2, 3, 8, 8, device="cuda")
    with pytest.raises(dm.DemagError) as ei:
        dm.demag_apply(plan.handle, m, 1.0, torch.empty_like(m), info=plan.info)
    assert ei.value.status == 1
    m1 = torch.zeros(1, 2, 3, 8, 8, device="cuda")
    with pytest.raises(dm.DemagError):
        dm.demag_apply(plan.handle, m1, 1.0, m1, info=plan.info)
    with pytest.raises(TypeError):
        plan.apply(m1.double(), 1.0)
    plan.close()


@pytest.mark.parametrize("nx,ny,th,prec", [(7, 5, (1.0, 0.5, 2.0), dm.PREC_SPLIT_TF32),
                                           (9, 6, tuple(np.round(np.linspace(0.6, 2.4, 10), 3)), dm.PREC_SPLIT_TF32),
                                           (9, 6, tuple(np.round(np.linspace(0.6, 2.4, 10), 3)), dm.PREC_SPLIT_BF16)])
def test_split_plan_tensor_matches_oracle_in_the_blocked_layout(nx, ny, th, prec):
    """A dense-product plan's stored tensor, decoded here from the documented
    blocked layout (8 x 8 layer blocks R <= C of M(i, j) = (t_i / t_0) N(i <- j),
    half h = b / 4 of row a of block (R, C) in 16-byte slot a ^ (C mod 4) ^ 4 h
    of half-block h, diagonal blocks mirrored
    with xz and yz negated, layers past L zero), equals
    the oracle's transformed kernels.  10 layers cross a block boundary.  A
    DEMAG_PREC_SPLIT_BF16 plan on path 7 stores each value as its BF16 split
    pair (hi << 16 | lo, hi + lo within 2^-18 of the value) and N_zz negated."""
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=prec, max_batch=1)
    info = plan.info
    packed = prec == dm.PREC_SPLIT_BF16
    assert info["path"] == 7 or not packed
    Px, Py, L = info["Px"], info["Py"], info["L"]
    Kx, Qy = Px // 2 + 1, Py // 2 + 1
    nb = (L + 7) // 8
    row = 64 * nb * (nb + 1) // 2
    out = torch.empty(Kx * Qy * 6 * row, dtype=torch.float32, device="cuda")
    dm.demag_plan_tensor(plan.handle, out)
    torch.cuda.synchronize()
    if packed:
        w = out.cpu().numpy().view(np.uint32)
        hi = (w & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
        lo = (w << np.uint32(16)).view(np.float32).astype(np.float64)
        T = (hi + lo).reshape(Kx, Qy, 6, row)
    else:
        T = out.cpu().numpy().astype(np.float64).reshape(Kx, Qy, 6, row)
    plan.close()
    ky_of_u = _stored_ky(Py, info["path"])
    K = reading_kernels(nx, ny, 2.0, 2.0, tuple(th))
    qs = np.arange(-(ny - 1), ny) % Py
    ps = np.arange(-(nx - 1), nx) % Px
    ref = {}
    for i in range(L):
        for j in range(i, L):
            Kp = np.zeros((6, Py, Px))
            Kp[:, qs[:, None], ps[None, :]] = K[i, j]
            S = np.fft.fft2(Kp) / (Px * Py)
            R = np.stack([S[0].real, S[1].real, S[2].real, S[3].real, S[4].imag, S[5].imag])
            ref[i, j] = np.transpose(R[:, ky_of_u, :Kx], (2, 1, 0))  # [kx, u, component]
    sign = np.array([1.0, 1.0, 1.0, 1.0, -1.0, -1.0])
    zz = np.array([1.0, 1.0, -1.0 if packed else 1.0, 1.0, 1.0, 1.0])
    exp = np.zeros_like(T)
    blk = 0
    for Rb in range(nb):
        for Cb in range(Rb, nb):
            for a in range(8):
                for b in range(8):
                    i, j = 8 * Rb + a, 8 * Cb + b
                    if i >= L or j >= L:
                        continue
                    h = b // 4  # half-row h of row a in slot a ^ (Cb mod 4) ^ 4h of half-block h
                    e = 64 * blk + 32 * h + 4 * (a ^ (Cb & 3) ^ (4 * h)) + (b & 3)
                    if i <= j:
                        exp[:, :, :, e] = zz * th[i] / th[0] * ref[i, j]
                    else:  # lower half of a diagonal block
                        exp[:, :, :, e] = zz * sign * th[j] / th[0] * ref[j, i]
            blk += 1
    sc = np.abs(exp).max()
    assert np.abs(T - exp).max() < (5e-6 if packed else 2e-6) * sc
