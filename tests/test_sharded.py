"""The frequency-sharded apply (paper_1910_07054_gb300/sharded.py) on the CPU:
its partitioning, and two gloo ranks (world size 2, 127.0.0.1) exchanging the
row spectra by all-to-all, against the same orchestration on one rank (bit for
bit) and against the oracle's hybrid field.

The local steps here are CPU stand-ins written from the oracle's pieces (numpy
FFTs and the oracle's kernel spectra); each treats every plane and every kx
column on its own, elementwise, so that splitting the work among ranks cannot
change a bit of the result."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

from paper_1910_07054_gb300.sharded import ShardedApply, even_ranges  # noqa: E402

STEPS = r"""
import os
import numpy as np
import torch
from oracle import demag as odm
from oracle import newell as onw
from paper_1910_07054_gb300 import inputs
from paper_1910_07054_gb300.sharded import ShardedApply

COMP = ((0, 3, 4), (3, 1, 5), (4, 5, 2))


def case():
    nx, ny, th, B, Ms = 10, 6, [1.0, 0.5, 2.0], 2, 8e5
    m = inputs.random_unit_vectors((B, len(th), ny, nx), seed=17)
    Kq = onw.layer_kernels(nx, ny, 2.0, 2.0, th, mode=onw.READING_D, full=False)
    Khat = odm.padded_kernel_spectra(odm.expand_quadrant(Kq))  # [L, L, 6, 2ny, 2nx]
    return nx, ny, th, B, Ms, m, Khat


def run(rank, world, dist):
    nx, ny, th, B, Ms, m, Khat = case()
    L = len(th)
    P, Kx = B * L * 3, nx + 1
    mp = torch.tensor(m.reshape(P, ny, nx))
    H = torch.zeros(P, ny, nx, dtype=torch.float64)
    Kt = torch.tensor(Khat[..., : nx + 1])  # kx = 0..nx of the rfft

    def rows_forward(p0, p1):
        x = torch.zeros(p1 - p0, ny, 2 * nx, dtype=torch.float64)
        x[:, :, :nx] = mp[p0:p1]
        return torch.fft.rfft(x, dim=2).transpose(1, 2).contiguous()  # [np, Kx, ny]

    def columns_slab(slab):
        k0, k1 = sa.slabs[rank]
        y = torch.zeros(P, k1 - k0, 2 * ny, dtype=torch.complex128)
        y[:, :, :ny] = slab
        Y = torch.fft.fft(y, dim=2).view(B, L, 3, k1 - k0, 2 * ny)
        out = torch.zeros_like(Y)
        for i in range(L):
            for a in range(3):
                for j in range(L):
                    for c in range(3):
                        out[:, i, a] += Kt[i, j, COMP[a][c], :, k0:k1].transpose(0, 1) * Y[:, j, c]
        slab[:] = torch.fft.ifft(out, dim=-1).reshape(P, k1 - k0, 2 * ny)[:, :, :ny]

    def rows_inverse(spec, p0, p1):
        H[p0:p1] = -Ms * torch.fft.irfft(spec.transpose(1, 2), n=2 * nx, dim=2)[:, :, :nx]

    stage = os.environ.get("DEMAG_STAGE_HOST") == "1"
    sa = ShardedApply(P, Kx, ny, rank, world, rows_forward, columns_slab, rows_inverse, dist, stage_host=stage)
    sa.apply()
    p0, p1 = sa.planes[rank]
    return H[p0:p1].numpy(), (p0, p1), sa
"""

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["DEMAG_ROOT"])
import numpy as np
import torch.distributed as dist
exec(os.environ["DEMAG_STEPS"])
world, rank = int(os.environ["WORLD_SIZE"]), int(os.environ["RANK"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%s" % os.environ["MASTER_PORT"], rank=rank,
                        world_size=world)
H, (p0, p1), sa = run(rank, world, dist)
parts = [None] * world
dist.all_gather_object(parts, (p0, p1, H.tobytes(), sa.bytes_exchanged(16)))
dist.barrier()
dist.destroy_process_group()
if rank == 0:
    full = np.concatenate([np.frombuffer(b, dtype=np.float64) for _, _, b, _ in sorted(parts)])
    np.save(os.environ["DEMAG_OUT"], full)
print(json.dumps({"rank": rank, "planes": [p0, p1], "slab": list(sa.slabs[rank]),
                  "sent": sa.bytes_exchanged(16)}))
"""


def test_even_ranges_cover_and_balance():
    for n in (0, 1, 5, 17, 513):
        for parts in (1, 2, 3, 8):
            r = even_ranges(n, parts)
            assert len(r) == parts and r[0][0] == 0 and r[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        even_ranges(4, 0)


def _single_rank():
    ns = {}
    exec(STEPS, ns)
    H, (p0, p1), sa = ns["run"](0, 1, None)
    nx, ny, th, B, Ms, m, Khat = ns["case"]()
    return H, m, Khat, Ms, sa


def test_single_rank_orchestration_matches_the_oracle():
    from oracle import demag as odm
    H, m, Khat, Ms, sa = _single_rank()
    ref = odm.hybrid(None, m, Ms, Khat=Khat)
    assert sa.bytes_exchanged(16) == 0
    assert np.linalg.norm(H.reshape(ref.shape) - ref) <= 1e-12 * np.linalg.norm(ref)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("stage_host", ["0", "1"])
def test_two_gloo_ranks_equal_one_rank_bit_for_bit(tmp_path, stage_host):
    """Both exchange modes: in place, and staged through host memory (the mode
    of gloo ranks whose spectra live on a GPU; here a copy of a host tensor)."""
    port = _free_port()
    out = str(tmp_path / "H.npy")
    procs = []
    for rank in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   DEMAG_ROOT=ROOT, DEMAG_STEPS=STEPS, DEMAG_OUT=out, DEMAG_STAGE_HOST=stage_host)
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    infos = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=240)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("gloo ranks did not finish")
        assert p.returncode == 0, e[-3000:]
        infos.append(json.loads(o.strip().splitlines()[-1]))
    infos.sort(key=lambda r: r["rank"])
    # 2 states x 3 layers x 3 components = 18 planes, 11 x-frequencies: disjoint halves
    assert infos[0]["planes"] == [0, 9] and infos[1]["planes"] == [9, 18]
    assert infos[0]["slab"] == [0, 6] and infos[1]["slab"] == [6, 11]
    assert all(r["sent"] > 0 for r in infos)
    H2 = np.load(out)
    H1, m, Khat, Ms, _ = _single_rank()
    assert np.array_equal(H2, H1.reshape(-1))  # bit for bit
