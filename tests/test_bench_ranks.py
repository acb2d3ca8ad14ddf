"""The multi-process host logic of bench.py on the CPU: two gloo ranks (world
size 2) on 127.0.0.1.  The path shards over independent magnetization states
with no data-path collective; the only exchange is the slowest rank's time,
which sets the whole-job value.  The reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys, time
sys.path.insert(0, os.environ["DEMAG_ROOT"])
import numpy as np
import torch.distributed as dist
import bench
from paper_1910_07054_gb300 import inputs

world, rank, local = bench.dist_env()
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%s" % os.environ["MASTER_PORT"],
                        rank=rank, world_size=world)
# each rank's own step time: the job is as slow as its slowest rank
step_ms = 1.0 + 0.5 * rank
T = bench.max_over_ranks(step_ms, dist)
value = bench.whole_job_value(world, 1, T)
# independent states per rank
m = inputs.mram_magnetization(16, 12, 3, seed=bench.rank_seed(rank), batch=1)
sums = [None] * world
dist.all_gather_object(sums, float(np.abs(m).sum() + 1e-3 * m[0, 0, 0].sum()))
# the reference arm: ranks other than 0 return at once, without work
ref_s = None
if rank != 0:
    t0 = time.perf_counter()
    out = bench.run_reference(None)
    ref_s = time.perf_counter() - t0
    assert out is None
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "T": T, "value": value, "sums": sums, "ref_s": ref_s}))
"""


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_share_only_the_slowest_time():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), DEMAG_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=240)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("gloo ranks did not finish")
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda r: r["rank"])
    for r in outs:
        assert r["T"] == 1.5                      # max over ranks, seen by both
        assert r["value"] == 2 / 1.5e-3           # both ranks' states in the slowest time
    assert outs[0]["sums"] == outs[1]["sums"]    # the gathered per-rank summaries agree
    assert outs[0]["sums"][0] != outs[0]["sums"][1]  # distinct states per rank
    assert outs[1]["ref_s"] is not None and outs[1]["ref_s"] < 1.0


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_value(1, 16, 2.0) == 8000.0
    assert bench.rank_seed(0) != bench.rank_seed(1)


def test_kernel_hash_ignores_comments_and_layout_only():
    sys.path.insert(0, ROOT)
    import bench
    a = 'int f(int x) {  // add one\n  return x + 1; /* done */ }\nconst char *s = "a // b";\n'
    b = 'int f(int x) {\n    return x + 1;\n}\n// a note\nconst char *s = "a // b";\n'
    c = 'int f(int x) { return x + 2; }\nconst char *s = "a // b";\n'
    d = 'int f(int x) { return x + 1; }\nconst char *s = "a //  b";\n'
    assert bench.code_only(a) == bench.code_only(b)      # comments and whitespace only
    assert bench.code_only(a) != bench.code_only(c)      # code
    assert bench.code_only(a) != bench.code_only(d)      # inside a literal
