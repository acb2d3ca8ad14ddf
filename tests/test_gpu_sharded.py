"""The frequency-sharded apply on the GPU.

The library's three sharded steps (demag_rows_forward, demag_columns_slab,
demag_rows_inverse) over ranks that each keep one kx slab of the tensor
(demag_plan_keep_slab) give demag_apply's field bit for bit: every column,
stored entry and row is computed by the same kernels, only split among the
ranks.  The ranks run here one after the other in one process, the exchanges
as device copies, for one to three ranks on each kernel family (1024-point
rows and columns with the tcgen05 BF16 and TF32 contractions and the
warp-level MMAs, 512-point rows with the generic columns, the FP32 and FP64
split paths); and as two gloo processes on the one GPU running ShardedApply
with host-staged exchanges, whose field is checked against the single-process
apply and against the oracle's hybrid."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch

import paper_1910_07054_gb300 as dm
from paper_1910_07054_gb300 import inputs
from paper_1910_07054_gb300.sharded import ShardedApply, even_ranges, gpu_steps

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# nx, ny, thicknesses, B, precision, path
CASES = [
    (300, 280, (1.0, 2.0, 0.5, 3.0), 2, dm.PREC_SPLIT_BF16, 7),
    (300, 280, (1.0, 2.0, 0.5, 3.0), 2, dm.PREC_SPLIT_TF32, 6),
    (300, 280, (1.0, 2.0, 0.5, 3.0), 2, dm.PREC_SPLIT_TF32, 4),
    (200, 140, (1.0, 2.0, 0.5, 1.5, 2.5, 1.0), 3, dm.PREC_SPLIT_TF32, 6),
    (40, 24, (1.0, 0.7, 2.0), 2, dm.PREC_FP32, 2),
    (40, 24, (1.0, 0.7, 2.0), 2, dm.PREC_FP64, 2),
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _plan(nx, ny, th, B, prec, path):
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=prec, max_batch=B)
    dm.demag_plan_set_path(plan.handle, path)
    plan.info = dm.demag_plan_info(plan.handle)
    return plan


def _sharded_in_one_process(nx, ny, th, B, prec, path, m, Ms, world):
    """Each rank's plan keeps its slab; the ranks' steps run in turn, the two
    all-to-alls as copies of device tensors."""
    L = len(th)
    P = B * L * 3
    cdt = torch.complex128 if prec == dm.PREC_FP64 else torch.complex64
    planes, H = None, torch.empty_like(m)
    plans, specs = [], []
    for r in range(world):
        plan = _plan(nx, ny, th, B, prec, path)
        Kx = plan.info["Px"] // 2 + 1
        planes, slabs = even_ranges(P, world), even_ranges(Kx, world)
        plan.keep_slab(*slabs[r])
        plans.append(plan)
        p0, p1 = planes[r]
        spec = torch.empty(p1 - p0, Kx, ny, dtype=cdt, device="cuda")
        specs.append(dm.demag_rows_forward(plan.handle, m, p0, p1, spec, info=plan.info))
    for r in range(world):
        k0, k1 = slabs[r]
        slab = torch.cat([s[:, k0:k1, :] for s in specs], dim=0).contiguous()
        dm.demag_columns_slab(plans[r].handle, slab, k0, k1, B, info=plans[r].info)
        for d, (q0, q1) in enumerate(planes):
            specs[d][:, k0:k1, :] = slab[q0:q1]
    for r in range(world):
        p0, p1 = planes[r]
        dm.demag_rows_inverse(plans[r].handle, specs[r], p0, p1, Ms, H, info=plans[r].info)
    torch.cuda.synchronize()
    assert dm.demag_wait_timeouts() == 0
    for plan in plans:
        plan.close()
    return H


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%d_L%d_B%d_p%d_path%d" % (c[0], c[1], len(c[2]), c[3],
                                                                                   c[4], c[5]))
def test_sharded_steps_equal_apply_bit_for_bit(case):
    nx, ny, th, B, prec, path = case
    dt = torch.float64 if prec == dm.PREC_FP64 else torch.float32
    m = torch.tensor(inputs.random_unit_vectors((B, len(th), ny, nx), seed=nx + B), dtype=dt, device="cuda")
    Ms = 8e5
    full = _plan(nx, ny, th, B, prec, path)
    assert full.info["path"] == path
    ref = full.apply(m, Ms)
    torch.cuda.synchronize()
    full.close()
    assert torch.isfinite(ref).all() and ref.abs().max() > 0
    for world in (1, 2, 3):
        H = _sharded_in_one_process(nx, ny, th, B, prec, path, m, Ms, world)
        assert torch.equal(H, ref), (world, (H - ref).abs().max().item())


def test_slab_plan_tensor_is_the_full_tensor_slab():
    nx, ny, th, B = 300, 280, (1.0, 2.0, 0.5, 3.0), 2
    full = _plan(nx, ny, th, B, dm.PREC_SPLIT_BF16, 7)
    nb = (len(th) + 7) // 8
    entry = 6 * nb * (nb + 1) // 2 * 64  # floats of one stored entry (8 x 8 layer blocks, R <= C)
    t_full = torch.empty(full.info["Px"] // 2 + 1, full.info["Py"] // 2 + 1, entry, device="cuda")
    dm.demag_plan_tensor(full.handle, t_full)
    full.keep_slab(100, 257)
    t_slab = torch.empty(157, *t_full.shape[1:], device="cuda")
    dm.demag_plan_tensor(full.handle, t_slab)
    torch.cuda.synchronize()
    # compared as bits: the BF16 plan's slots hold split pairs, not floats
    assert torch.equal(t_slab.view(torch.int32), t_full[100:257].view(torch.int32))


def test_slab_plan_restrictions():
    nx, ny, th, B = 40, 24, (1.0, 0.7, 2.0), 2
    m = torch.zeros(B, 3, 3, ny, nx, device="cuda")
    plan = _plan(nx, ny, th, B, dm.PREC_FP32, 2)
    Kx = plan.info["Px"] // 2 + 1
    with pytest.raises(dm.DemagError):
        plan.keep_slab(3, 3)  # empty range
    with pytest.raises(dm.DemagError):
        plan.keep_slab(0, Kx + 1)
    plan.keep_slab(2, 7)
    with pytest.raises(dm.DemagError):
        plan.apply(m, 1.0)  # the plan holds only a slab
    with pytest.raises(dm.DemagError):
        plan.keep_slab(2, 7)  # already a slab
    spec = torch.zeros(B * 9, 6, ny, dtype=torch.complex64, device="cuda")
    with pytest.raises(dm.DemagError):
        dm.demag_columns_slab(plan.handle, spec, 1, 7, B)  # outside the kept slab
    dm.demag_columns_slab(plan.handle, spec[:, :5].contiguous(), 2, 7, B)  # zero in, zero out
    with pytest.raises(ValueError):
        dm.demag_rows_forward(plan.handle, m, 0, B * 9 + 1,
                              torch.empty(B * 9 + 1, Kx, ny, dtype=torch.complex64, device="cuda"))
    fused = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_FP32, max_batch=B)
    if fused.info["path"] != 2:
        with pytest.raises(dm.DemagError):
            fused.keep_slab(0, 4)  # off the split path
    torch.cuda.synchronize()
    plan.close()
    fused.close()


RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["DEMAG_ROOT"])
import numpy as np
import torch
import torch.distributed as dist
import paper_1910_07054_gb300 as dm
from paper_1910_07054_gb300 import inputs
from paper_1910_07054_gb300.sharded import ShardedApply, even_ranges, gpu_steps
world, rank = int(os.environ["WORLD_SIZE"]), int(os.environ["RANK"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%s" % os.environ["MASTER_PORT"], rank=rank,
                        world_size=world)
torch.cuda.set_device(0)
nx, ny, th, B, Ms = 300, 280, (1.0, 2.0, 0.5, 3.0), 2, 8e5
L = len(th)
m = torch.tensor(inputs.random_unit_vectors((B, L, ny, nx), seed=5), dtype=torch.float32, device="cuda")
H = torch.zeros_like(m)
plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_SPLIT_BF16, max_batch=B)
P, Kx = B * L * 3, plan.info["Px"] // 2 + 1
k0, k1 = even_ranges(Kx, world)[rank]
plan.keep_slab(k0, k1)
steps = gpu_steps(plan, m, H, B, Ms, k0, k1)
sa = ShardedApply(P, Kx, ny, rank, world, *steps, dist=dist, stage_host=True)
sa.apply()
torch.cuda.synchronize()
p0, p1 = sa.planes[rank]
mine = H.view(P, ny, nx)[p0:p1].cpu().numpy()
parts = [None] * world
dist.all_gather_object(parts, (p0, p1, mine.tobytes()))
dist.barrier()
dist.destroy_process_group()
if rank == 0:
    full = np.concatenate([np.frombuffer(b, dtype=np.float32) for _, _, b in sorted(parts)])
    np.save(os.environ["DEMAG_OUT"], full)
print(json.dumps({"rank": rank, "planes": [p0, p1], "slab": [k0, k1], "timeouts": dm.demag_wait_timeouts(),
                  "sent": sa.bytes_exchanged(8)}))
"""


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_on_the_gpu_equal_one_process(tmp_path):
    port = _free_port()
    out = str(tmp_path / "H.npy")
    procs = []
    for rank in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   DEMAG_ROOT=ROOT, DEMAG_OUT=out)
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    infos = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("gloo ranks did not finish")
        assert p.returncode == 0, e[-3000:]
        infos.append(json.loads(o.strip().splitlines()[-1]))
    infos.sort(key=lambda r: r["rank"])
    # 2 states x 4 layers x 3 components = 24 planes; Px = 1024: 513 x-frequencies
    assert infos[0]["planes"] == [0, 12] and infos[1]["planes"] == [12, 24]
    assert infos[0]["slab"] == [0, 257] and infos[1]["slab"] == [257, 513]
    assert all(r["timeouts"] == 0 and r["sent"] > 0 for r in infos)
    H2 = torch.tensor(np.load(out)).view(2, 4, 3, 280, 300)

    nx, ny, th, B, Ms = 300, 280, (1.0, 2.0, 0.5, 3.0), 2, 8e5
    m = inputs.random_unit_vectors((B, len(th), ny, nx), seed=5)
    plan = dm.Plan(nx, ny, 2.0, 2.0, th, precision=dm.PREC_SPLIT_BF16, max_batch=B)
    ref = plan.apply(torch.tensor(m, dtype=torch.float32, device="cuda"), Ms).cpu()
    plan.close()
    assert torch.equal(H2, ref)
    # and the field itself against the oracle's hybrid on one target layer of one state
    from oracle import demag as odm
    from oracle import newell as onw
    want = odm.hybrid_targets(lambda i, j: onw.pair_kernel(nx, ny, 2.0, 2.0, list(th), i, j), m[1], Ms, [2])[2]
    got = H2[1, 2].double().numpy()
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)
