#!/usr/bin/env python3
"""Benchmark of the hybrid demagnetization field (Eq. FFT_v2) on GB300.

One step = one application of the method to a batch of magnetization states
through the C ABI on device-resident inputs.  The headline workload is the
largest single-GPU stack: 512 x 512 cells of 2 x 2 nm, 64 layers with
thicknesses uniform in [0.5, 3] nm (seed 0), 16 random states per apply, float
FFTs and the split-precision contraction (three TF32 passes, float
accumulation) on the tcgen05 tensor cores.  Its inputs (3.2 GB of m, a 13.1 GB
tensor) are far larger than the 129 MB L2, so consecutive steps start cold.
Steps are timed with CUDA events on the launching stream.

Beside it: the 256 x 256 x 8 MRAM-like stack as a full block of its own (a
256 MB buffer written between its steps), the split-precision variants, the
differentiation and the surrogate workloads, and the oracle on the host cores.

Prints one JSON line (rank 0).  Under torchrun each rank evaluates its own
independently seeded states on its own GPU (replicas, weak scaling) and the
slowest rank's time sets the value.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "demag evals/s and Gcell-layers/s at ≤1e-5 rel L2 vs FP64 oracle; % HBM peak"
HEADLINE = "scale512"
WORKLOAD = "mram256"
FLUSH_BYTES = 256 << 20
HBM_FALLBACK_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--cpu-budget", type=float, default=20.0,
                   help="seconds of oracle evaluation for the 256x256x8 CPU baseline sample")
    p.add_argument("--no-allcore", action="store_true", help="skip the all-core oracle timing")
    p.add_argument("--no-parity", action="store_true", help="skip the oracle field comparison")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--batched-only", action="store_true",
                   help="run only the batched split-precision measurement and print its JSON")
    p.add_argument("--batched-n", type=int, default=512,
                   help="in-plane cells per side of the batched measurement (smaller for profiling)")
    p.add_argument("--batched-layers", type=int, default=64,
                   help="layers of the batched measurement (the first of its 64; fewer for profiling)")
    p.add_argument("--batched-paths", default="6,7,4,3",
                   help="contraction paths of the batched measurement (comma separated)")
    p.add_argument("--hysteresis-only", action="store_true",
                   help="run only the Sec. 4 MRAM free-layer hysteresis and print its JSON")
    p.add_argument("--grad-only", action="store_true",
                   help="run only the differentiation measurement and print its JSON")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the 256x256x8 block, the split-precision variants, the differentiation and "
                        "the surrogate measurements")
    p.add_argument("--sweep-only", action="store_true",
                   help="run only the hybrid vs 3D-FFT nz sweep at 256x256 and print its JSON")
    p.add_argument("--mram-only", action="store_true",
                   help="run only the 256x256x8 block (device timing) and print its JSON")
    return p.parse_args()


def workload():
    from paper_1910_07054_gb300 import inputs
    c = inputs.CONFIGS[WORKLOAD]
    th = [float(t) for t in inputs.thicknesses(WORKLOAD)]
    desc = ("MRAM-like stack: %dx%d cells of %gx%g nm, %d layers of %s nm, batch %d; odd layers two "
            "+-z half-plane domains, even layers seeded random unit vectors; Ms = %g A/m; float32 "
            "FFTs and contraction, float64 tensor set-up"
            % (c["nx"], c["ny"], c["dx"], c["dy"], len(th), th, c["batch"], inputs.MS_DEFAULT))
    return c, th, desc


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(rank):
    """Seed of a rank's magnetization states: every rank evaluates its own
    independent states (the path shards over states, no data-path collective)."""
    return rank


def max_over_ranks(value, dist=None, device="cpu"):
    """The slowest rank's value (all ranks receive it); the value itself on one
    process.  NCCL ranks pass device="cuda", gloo ranks the CPU."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, batch_per_rank, step_ms):
    """Evaluations per second of the whole job: every rank's states in the time
    of the slowest rank's step."""
    return world * batch_per_rank / (step_ms * 1e-3)


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the GPU works."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = max((num(r[2]) for r in rows if num(r[2]) is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = sorted(v for v in sm if smax and v > 0.5 * smax) or sorted(sm)
        med = loaded[len(loaded) // 2] if loaded else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows)}


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = json.load(fh).get("hbm_gbs")
        if v:
            return float(v), "measured"
    except (OSError, ValueError):
        pass
    return HBM_FALLBACK_GBS, "fallback"


def code_only(text):
    """C/C++ source with its comments (// to end of line, /* ... */) and every
    run of whitespace outside literals reduced to one space, string and
    character literals kept: what the compiled kernels depend on."""
    out, i, n = [], 0, len(text)

    def space():
        if out and out[-1] != " ":
            out.append(" ")

    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
            space()
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            space()
        elif c.isspace():
            i += 1
            space()
        else:
            out.append(c)
            i += 1
    return "".join(out)


def kernel_source_hash(names=("apply.cu", "apply512.cu", "fft.cuh", "fft8.cuh"), read=None):
    """Hash of kernel sources, comments excluded (a comment edit does not change
    the counters recorded for them)."""
    h = hashlib.sha256()
    for name in names:
        if read is None:
            with open(os.path.join(ROOT, "paper_1910_07054_gb300", "csrc", name), encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(name)
        h.update(code_only(text).encode("utf-8"))
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of that kernel; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = rec.get("kernels", {}).get(kernel)
    if ent is None or ent.get("source_hash") != kernel_source_hash(tuple(ent.get("sources", ()))):
        return None
    return ent.get("dram_bytes_per_launch")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ---- oracle (host cores) --------------------------------------------------------

def oracle_setup(c, th):
    """Oracle spectra of the 256 x 256 x 8 workload's layer kernels (float64, CPU)."""
    from oracle import demag as odm
    from oracle import newell as onw
    Kq = onw.layer_kernels(c["nx"], c["ny"], c["dx"], c["dy"], th, mode=onw.READING_D, full=False)
    return odm.padded_kernel_spectra(odm.expand_quadrant(Kq))


def oracle_timed(Khat, m_np, Ms, budget_s, max_evals):
    """Times whole oracle evaluations of the workload until budget_s is spent."""
    from oracle import demag as odm
    times, H = [], None
    t_start = time.perf_counter()
    while len(times) < max_evals:
        t0 = time.perf_counter()
        H = odm.hybrid(None, m_np, Ms, Khat=Khat)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s:
            break
    return times, H


def headline_workload():
    from paper_1910_07054_gb300 import inputs
    c = inputs.CONFIGS[HEADLINE]
    th = [float(t) for t in inputs.thicknesses(HEADLINE)]
    desc = ("layer scaling + batch: %dx%d cells of %gx%g nm, %d layers with thicknesses uniform in [%g, %g] nm "
            "(seed %d), %d random unit-vector states per apply (normalised N(0,1) triples); Ms = %g A/m; float32 "
            "FFTs, split-precision contraction (3xBF16 passes, float accumulate) on the tcgen05 tensor cores, "
            "float64 tensor set-up"
            % (c["nx"], c["ny"], c["dx"], c["dy"], len(th), c["thickness_range"][0], c["thickness_range"][1],
               c["seed"], c["batch"], inputs.MS_DEFAULT))
    return c, th, desc


def headline_config(c, th, desc, world, info=None):
    cfg = {"workload": desc, "nx": c["nx"], "ny": c["ny"], "layers": len(th), "batch_per_gpu": c["batch"],
           "padded_fft": [info["Px"], info["Py"]] if info else [2 * c["nx"], 2 * c["ny"]],
           "l2": "inputs larger than L2 (m 3.2 GB, stored tensor 14.6 GB per step against a 129 MB L2); no flush",
           "parallelism": "replicas" if world > 1 else "single GPU"}
    return cfg


# The sampled oracle evaluation of the headline workload: one target layer of
# one state, Eq. FFT_v2 pair by pair (oracle.demag.hybrid_targets as it
# stands: forward FFTs of the state's 3L source planes, per source layer the
# spectra of the pair kernel and the 3x3 products, inverse FFT of the target's
# three planes).  The pair kernels of that target row are evaluated once
# beforehand (tensor set-up, not timed).  A whole state is L such target
# layers, so evals/s = 1 / (L * sample time); this overstates the oracle's cost
# slightly (the source FFTs would be shared between targets) and is stated so.
SAMPLE_TARGET = 37


def headline_pair_kernels(c, th, target=SAMPLE_TARGET):
    import numpy as np
    from oracle import newell as onw
    return np.stack([onw.pair_kernel(c["nx"], c["ny"], c["dx"], c["dy"], th, target, j)
                     for j in range(len(th))])


def headline_oracle_sample(pk, m_state, Ms, target=SAMPLE_TARGET):
    from oracle import demag as odm
    t0 = time.perf_counter()
    H = odm.hybrid_targets(lambda i, j: pk[j], m_state, Ms, [target])[target]
    return time.perf_counter() - t0, H


def _allcore_worker(job):
    """One process of the all-core oracle timing (spawned): the headline sample
    on its own state, started at a common wall-clock instant."""
    import numpy as np
    from oracle import demag as odm
    pk_path, m_path, state, Ms, target, start_at = job
    pk = np.load(pk_path, mmap_mode="r")
    m = np.array(np.load(m_path, mmap_mode="r")[state])
    while time.time() < start_at:
        time.sleep(0.005)
    t0 = time.time()
    odm.hybrid_targets(lambda i, j: np.asarray(pk[j]), m, Ms, [target])
    return t0, time.time()


def headline_oracle_allcore(pk, m_np, Ms, L):
    """The headline sample run concurrently by one spawned process per core (as
    many as the host's free memory allows, about 6 GB each): evals/s of the
    whole host."""
    import multiprocessing as mp
    import shutil

    import numpy as np
    ncpu = os.cpu_count() or 1
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 0
    nproc = max(1, min(ncpu, int(avail // (6 << 30))))
    base = "/dev/shm" if os.path.isdir("/dev/shm") else None
    tmp = tempfile.mkdtemp(prefix="demag_oracle_", dir=base)
    try:
        pk_path, m_path = os.path.join(tmp, "pk.npy"), os.path.join(tmp, "m.npy")
        np.save(pk_path, pk)
        np.save(m_path, m_np[:min(nproc, m_np.shape[0])])
        ctx = mp.get_context("spawn")
        with ctx.Pool(nproc) as pool:
            pool.map(abs, range(nproc))  # workers started and imported before the clock
            start = time.time() + 2.0
            jobs = [(pk_path, m_path, k % min(nproc, m_np.shape[0]), Ms, SAMPLE_TARGET, start)
                    for k in range(nproc)]
            spans = pool.map(_allcore_worker, jobs)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    wall = max(t1 for _, t1 in spans) - min(t0 for t0, _ in spans)
    return {"value": nproc / (L * wall), "unit": "evals/s", "cores": nproc, "kind": "oracle",
            "host_cpus": ncpu,
            "sample": "%d concurrent spawned processes, each one target layer of one state (the single-thread "
                      "sample), %.1f s wall; evals/s = processes / (%d layers x wall)" % (nproc, wall, L)}


def run_reference(args):
    """The oracle (float64 numpy + C) on the host cores for the headline
    workload, sampled: each step is one target layer of one state (see
    headline_oracle_sample), at most --steps samples after at most one warm-up
    sample, bounded to about a minute."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from paper_1910_07054_gb300 import inputs
    c, th, desc = headline_workload()
    L = len(th)
    m = inputs.random_unit_vectors((1, L, c["ny"], c["nx"]), seed=0)
    t0 = time.perf_counter()
    pk = headline_pair_kernels(c, th)
    setup_s = time.perf_counter() - t0
    warm = min(args.warmup, 1)
    for _ in range(warm):
        headline_oracle_sample(pk, m[0], inputs.MS_DEFAULT)
    times = []
    t_start = time.perf_counter()
    while len(times) < max(args.steps, 1):
        times.append(headline_oracle_sample(pk, m[0], inputs.MS_DEFAULT)[0])
        if time.perf_counter() - t_start > 60.0:
            break
    per = float(np.mean(times))
    value = 1.0 / (L * per)
    sample = ("%d samples (of %d steps requested) after %d warm-up, each one target layer of one state: oracle "
              "float64 hybrid_targets (numpy FFT, single thread) over the 64 source layers; evals/s = 1 / (64 x "
              "sample time); pair kernels of the target row evaluated beforehand in %.1f s, not timed"
              % (len(times), args.steps, warm, setup_s))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": 0,
            "steps": len(times), "warmup": warm, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(headline_config(c, th, desc, 1), parallelism="host cores"),
            "gcell_layers_per_s": c["nx"] * c["ny"] * L * value / 1e9,
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- GPU measurements ---------------------------------------------------------------

COMPRESS_TOL = 1e-8  # demag_plan_compress tolerance of the compressed-tensor measurement


def info_tensor_bytes(info):
    """Bytes of a dense-product plan's uncompressed (blocked) tensor."""
    nb = (info["L"] + 7) // 8
    return (info["Px"] // 2 + 1) * (info["Py"] // 2 + 1) * 6 * 64 * nb * (nb + 1) // 2 * 4


def split_stage_names(info):
    r = "1024" if info["Px"] == 1024 else ""
    cfwd = "k_columns_forward1024" if info["Py"] == 1024 else "k_columns_forward"
    cinv = "k_columns_inverse1024" if info["Py"] == 1024 else "k_columns_inverse"
    contract = {6: "k_contract_tc5<false>", 7: "k_contract_tc5<true>", 4: "k_contract_tc",
                3: "k_contract_gemm"}.get(info["path"], "k_contract")
    return ["k_rows_forward" + r, cfwd, contract, cinv, "k_rows_inverse" + r]


def split_stage_bytes(info, B):
    """Algorithmic bytes of the five split-path kernels (float32): field, row
    spectrum [B][L][3][Kx][ny], column spectrum [Kx][Py][B][L][3] and the
    compact tensor (6 reals per stored pair and entry, Kx x (Py/2+1) entries)."""
    L, nx, ny = info["L"], info["nx"], info["ny"]
    Kx, Py, Qy = info["Px"] // 2 + 1, info["Py"], info["Py"] // 2 + 1
    field = B * L * 3 * ny * nx * 4
    spec = B * L * 3 * Kx * ny * 8
    spec2 = B * L * 3 * Kx * Py * 8
    tensor = Kx * Qy * info["npairs"] * 6 * 4
    return [field + spec, spec + spec2, 2 * spec2 + tensor, spec2 + spec, spec + field], field, tensor


def time_steps(run, steps, stream, before=None):
    """CUDA-event time of each of `steps` calls of run(), on `stream`."""
    import numpy as np
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        if before is not None:
            before(k)
        starts[k].record(stream)
        run()
        ends[k].record(stream)
    torch.cuda.synchronize()
    return np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])


def mram_block(args, world, rank, dist, peaks, with_oracle):
    """The 256 x 256 x 8 MRAM-like stack (float32, one state per apply): device
    timing with a 256 MB L2 flush between steps, per-kernel times and the
    roofline of the dominant kernel, end to end through pinned host buffers,
    parity and the single-thread oracle."""
    import numpy as np
    import torch

    import paper_1910_07054_gb300 as dm
    from paper_1910_07054_gb300 import inputs
    c, th, desc = workload()
    nx, ny, L, B = c["nx"], c["ny"], len(th), c["batch"]
    Ms = inputs.MS_DEFAULT
    m_np = inputs.mram_magnetization(nx, ny, L, seed=rank_seed(rank), batch=B)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plan = dm.Plan(nx, ny, c["dx"], c["dy"], th, precision=dm.PREC_FP32, max_batch=B)
    plan_s = time.perf_counter() - t0
    info = plan.info
    m = torch.tensor(m_np, dtype=torch.float32, device="cuda")
    H = torch.empty_like(m)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    steps = max(args.steps, 20)
    for k in range(max(args.warmup, 3)):
        flush.fill_(float(k))
        dm.demag_apply(plan.handle, m, Ms, H, stream, info)
    torch.cuda.synchronize()
    step_ms = time_steps(lambda: dm.demag_apply(plan.handle, m, Ms, H, stream, info), steps, stream,
                         before=lambda k: flush.fill_(float(k)))
    T = max_over_ranks(float(step_ms.mean()), dist, "cuda")
    value = whole_job_value(world, B, T)
    stage = np.zeros(3)
    nk = min(steps, 200)
    for k in range(nk):
        flush.fill_(float(k))
        stage += np.array(dm.demag_apply_timed(plan.handle, m, Ms, H, stream, info)[:3])
    stage /= nk
    # end to end on page-locked host buffers, every evaluation copying its state
    # in and its field out.  Streamed (the value): demag_apply_host_async on two
    # alternating buffer sets, one evaluation's copies overlapping another's
    # kernels; one call at a time: demag_apply_host (the kernels read m and
    # write H over the host link), synchronised every call
    H_dev = H.clone().cpu()
    mh = [torch.tensor(m_np, dtype=torch.float32).pin_memory() for _ in range(2)]
    Hh = [torch.empty_like(mh[0]).pin_memory() for _ in range(2)]
    ne = min(steps, 200)
    for k in range(2):
        dm.demag_apply_host_async(plan.handle, mh[k], Ms, Hh[k], stream, info)
    dm.demag_apply_host_wait(plan.handle, stream)
    if dist:
        dist.barrier()
    e0 = time.perf_counter()
    for k in range(ne):
        dm.demag_apply_host_async(plan.handle, mh[k & 1], Ms, Hh[k & 1], stream, info)
    dm.demag_apply_host_wait(plan.handle, stream)
    e2e_s = max_over_ranks((time.perf_counter() - e0) / ne, dist, "cuda")
    e2e_match = bool(torch.equal(Hh[0], H_dev) and torch.equal(Hh[1], H_dev))
    dm.demag_apply_host(plan.handle, mh[0], Ms, Hh[0], stream, info)
    e0 = time.perf_counter()
    for _ in range(ne):
        dm.demag_apply_host(plan.handle, mh[0], Ms, Hh[0], stream, info)
    sync_s = max_over_ranks((time.perf_counter() - e0) / ne, dist, "cuda")
    e2e_match = e2e_match and bool(torch.equal(Hh[0], H_dev))
    Kx, Qy, npairs = info["Px"] // 2 + 1, info["Py"] // 2 + 1, info["npairs"]
    field = B * L * 3 * ny * nx * 4
    spec = B * L * 3 * Kx * ny * 8
    tensor = Kx * npairs * 6 * Qy * 4
    stage_bytes = [field + spec, 2 * spec + tensor, spec + field]
    r8 = "8" if info["Px"] == 512 else ""
    col = "k_columns_fused"
    if info["path"] == 5:
        col = "k_columns_ring8" if L <= 11 else "k_columns_fused8"
    names = ["k_rows_forward" + r8, col, "k_rows_inverse" + r8]
    dom = int(np.argmax(stage))
    peak = float(peaks.get("hbm_gbs") or HBM_FALLBACK_GBS)
    achieved = stage_bytes[dom] / (stage[dom] * 1e-3) / 1e9
    out = {"workload": desc, "nx": nx, "ny": ny, "layers": L, "batch": B,
           "l2": "256 MB buffer written between timed steps (cold L2 per step)", "steps": steps,
           "value": value, "unit": "evals/s", "ms_per_step": T, "gcell_layers_per_s": nx * ny * L * value / 1e9,
           "hbm_frac_min_bytes": ((2 * field + tensor) / (T * 1e-3) / 1e9) / peak,
           "kernels_ms": dict(zip(names, [float(v) for v in stage])),
           "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak,
                        "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback", "unit": "GB/s",
                        "frac": achieved / peak, "traffic": recorded_traffic(names[dom]),
                        "algorithmic_bytes": stage_bytes[dom]},
           "e2e": {"value": whole_job_value(world, B, e2e_s * 1e3), "unit": "evals/s",
                   "h2d_bytes_per_step": field, "d2h_bytes_per_step": field,
                   "how": "demag_apply_host_async on page-locked buffers, %d consecutive evaluations (each "
                          "copies its state in and its field out, overlapping another's kernels), then "
                          "demag_apply_host_wait; no L2 flush between evaluations (the 57 MB tensor stays in "
                          "L2, as in a loop of evaluations), unlike the device timing's cold L2 per step" % ne,
                   "one_call_at_a_time": {"value": whole_job_value(world, B, sync_s * 1e3), "unit": "evals/s",
                                          "how": "demag_apply_host on device-mapped page-locked buffers, "
                                                 "synchronised every call (%d calls)" % ne},
                   "field_equals_device_run": e2e_match},
           "plan_create_s": plan_s, "rel_l2_vs_oracle": None, "cpu_baseline": None}
    if rank == 0 and with_oracle:
        Khat = oracle_setup(c, th)
        times, H_ref = oracle_timed(Khat, m_np, Ms, args.cpu_budget, 1000)
        out["cpu_baseline"] = {"value": B / float(np.mean(times)), "unit": "evals/s", "cores": 1, "kind": "oracle",
                               "sample": "%d whole evaluations of the workload, oracle float64 hybrid (numpy FFT, "
                                         "single thread), tensor set-up not timed" % len(times)}
        out["rel_l2_vs_oracle"] = float(np.linalg.norm(H.double().cpu().numpy() - H_ref) / np.linalg.norm(H_ref))
    plan.close()
    return out


def batched_measurement(steps, peaks, n=512, layers=64, paths=(6, 7, 4, 3)):
    """512 x 512 cells (n x n if given), 64 layers, 16 states per apply: the
    split-precision contraction on the tcgen05 tensor cores (path 6, the
    DEMAG_PREC_SPLIT_TF32 plan's default), with warp-level MMAs (path 4) and the
    same products on the FP32 cores (path 3), all on one plan; and path 7 on a
    DEMAG_PREC_SPLIT_BF16 plan (its tensor stored as BF16 split pairs), built
    when path 7 is asked for.  Same data movement throughout."""
    import numpy as np
    import torch

    import paper_1910_07054_gb300 as dm
    from paper_1910_07054_gb300 import inputs
    c = inputs.CONFIGS["scale512"]
    th = [float(t) for t in inputs.thicknesses("scale512")][:layers]
    nx, ny, B, L = n, n, c["batch"], len(th)
    t0 = time.perf_counter()
    plan = dm.Plan(nx, ny, c["dx"], c["dy"], th, precision=dm.PREC_SPLIT_TF32, max_batch=B)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    m = torch.tensor(inputs.random_unit_vectors((B, L, ny, nx), seed=0), dtype=torch.float32, device="cuda")
    H = torch.empty_like(m)
    out = {"workload": "%dx%d cells of 2x2 nm, %d layers (t ~ U[0.5, 3] nm, seed 0), 16 random "
                       "states per apply; inputs (%.2f GB)" % (nx, ny, L, B * L * 3 * nx * ny * 4 / 1e9),
           "plan_create_s": build_s}
    fields = {}
    names = {4: "tensor_cores_3xtf32", 6: "tcgen05_3xtf32", 7: "tcgen05_3xbf16", 3: "fp32_cores"}
    plan_bf16 = None
    for path in paths:
        name = names[path]
        if path == 7:
            if plan_bf16 is None:
                plan_bf16 = dm.Plan(nx, ny, c["dx"], c["dy"], th, precision=dm.PREC_SPLIT_BF16, max_batch=B)
            use = plan_bf16
        else:
            use = plan
            dm.demag_plan_set_path(use.handle, path)
        info = dm.demag_plan_info(use.handle)
        if info["path"] != path:  # e.g. odd L: the tcgen05 kernel does not hold the plan
            out[name] = {"skipped": "the plan runs path %d, not %d" % (info["path"], path)}
            continue
        dm.demag_apply(use.handle, m, inputs.MS_DEFAULT, H, info=info)
        st = np.mean([dm.demag_apply_timed(use.handle, m, inputs.MS_DEFAULT, H, info=info)
                      for _ in range(steps)], axis=0)
        total = float(st[0] + st[1] + st[2])
        fields[path] = H.clone()
        flops = 36.0 * L * L * B * (nx + 1) * (2 * ny)  # useful contraction flops per apply
        out[name] = {"states_per_s": B / (total * 1e-3), "ms_per_apply": total,
                     "kernels_ms": {"rows_forward": float(st[0]), "columns_forward": float(st[3]),
                                    "contraction": float(st[4]), "columns_inverse": float(st[5]),
                                    "rows_inverse": float(st[2])},
                     "contraction_tflops_useful": flops / (st[4] * 1e-3) / 1e12}
    bf16_peak = float(peaks.get("bf16_tflops", 1894.6))
    for name in ("tensor_cores_3xtf32", "tcgen05_3xtf32", "tcgen05_3xbf16"):
        if name not in out or "skipped" in out[name]:
            continue
        tc = out[name]
        bf = name == "tcgen05_3xbf16"
        peak = bf16_peak if bf else bf16_peak * (1.1 / 2.25)
        tc["tensor_pipe"] = {"bound": "tensor", "achieved": 3 * tc["contraction_tflops_useful"],
                             "peak": peak, "unit": "TFLOP/s",
                             "frac": 3 * tc["contraction_tflops_useful"] / peak,
                             "note": ("BF16 issue rate (3 passes per useful flop) against the measured bf16 burst "
                                      "peak") if bf else
                                     ("TF32 issue rate (3 passes per useful flop) against the measured bf16 burst "
                                      "peak x nominal tf32/bf16 ratio (1.1/2.25)")}
    if 3 in fields:
        ref = fields[3].double()
        for p in fields:
            if p != 3:
                out["rel_l2_%s_vs_fp32_cores" % names[p]] = float(
                    torch.linalg.vector_norm(fields[p].double() - ref) / torch.linalg.vector_norm(ref))
        if 6 in fields:
            out["speedup_tcgen05_vs_fp32_cores"] = out["fp32_cores"]["ms_per_apply"] / \
                out["tcgen05_3xtf32"]["ms_per_apply"]
    plan.close()
    if plan_bf16 is not None:
        plan_bf16.close()
    return out


def headline_measurement(args, world, rank, dist, peaks):
    """The headline: 512 x 512 x 64 layers x 16 states, split-precision plan on
    its default path (tcgen05 contraction)."""
    import numpy as np
    import torch

    import paper_1910_07054_gb300 as dm
    from paper_1910_07054_gb300 import inputs
    c, th, desc = headline_workload()
    nx, ny, L, B = c["nx"], c["ny"], len(th), c["batch"]
    Ms = inputs.MS_DEFAULT
    m_np = inputs.random_unit_vectors((B, L, ny, nx), seed=rank_seed(rank))
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plan = dm.Plan(nx, ny, c["dx"], c["dy"], th, precision=dm.PREC_SPLIT_BF16, max_batch=B)
    plan_s = time.perf_counter() - t0
    info = plan.info
    m = torch.tensor(m_np, dtype=torch.float32, device="cuda")
    H = torch.empty_like(m)
    run = lambda: dm.demag_apply(plan.handle, m, Ms, H, stream, info)  # noqa: E731
    for _ in range(max(args.warmup, 3)):
        run()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_ms = time_steps(run, args.steps, stream)
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    T = max_over_ranks(float(step_ms.mean()), dist, "cuda")
    value = whole_job_value(world, B, T)
    nk = min(args.steps, 10)
    stage = np.mean([dm.demag_apply_timed(plan.handle, m, Ms, H, stream, info) for _ in range(nk)], axis=0)
    kernels_ms = [float(stage[0]), float(stage[3]), float(stage[4]), float(stage[5]), float(stage[2])]
    names = split_stage_names(info)
    sbytes, field, tensor = split_stage_bytes(info, B)
    dom = int(np.argmax(kernels_ms))
    peak = float(peaks.get("hbm_gbs") or HBM_FALLBACK_GBS)
    achieved = sbytes[dom] / (kernels_ms[dom] * 1e-3) / 1e9
    flops = 36.0 * L * L * B * (nx + 1) * (2 * ny)
    bf16_peak = float(peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops") or 1700.0)
    H_gpu = H.clone()
    # end to end through the host entry points on page-locked buffers: every step
    # copies its 16 states in and its 16 fields out.  Streamed: consecutive
    # steps overlap one step's copies with another's kernels (two sets of host
    # buffers alternate); one call at a time: demag_apply_host, synchronised
    mh = [torch.from_numpy(m_np.astype(np.float32)).pin_memory() for _ in range(2)]
    Hh = [torch.empty_like(mh[0]).pin_memory() for _ in range(2)]
    ne = max(1, min(args.steps, 50))  # streamed steps: the pipeline's fill and drain amortise
    ns = max(1, min(args.steps, 10))  # synchronised calls
    for k in range(2):
        dm.demag_apply_host_async(plan.handle, mh[k], Ms, Hh[k], stream, info)
    dm.demag_apply_host_wait(plan.handle, stream)
    if dist:
        dist.barrier()
    e0 = time.perf_counter()
    for k in range(ne):
        dm.demag_apply_host_async(plan.handle, mh[k & 1], Ms, Hh[k & 1], stream, info)
    dm.demag_apply_host_wait(plan.handle, stream)
    e2e_s = max_over_ranks((time.perf_counter() - e0) / ne, dist, "cuda")
    e2e_match = bool(torch.equal(Hh[0], H_gpu.cpu()) and torch.equal(Hh[1], H_gpu.cpu()))
    dm.demag_apply_host(plan.handle, mh[0], Ms, Hh[0], stream, info)
    e0 = time.perf_counter()
    for _ in range(ns):
        dm.demag_apply_host(plan.handle, mh[0], Ms, Hh[0], stream, info)
    sync_s = max_over_ranks((time.perf_counter() - e0) / ns, dist, "cuda")
    e2e_match = e2e_match and bool(torch.equal(Hh[0], H_gpu.cpu()))
    del mh, Hh
    # the same plan with its tensor block-compressed (demag_plan_compress): the
    # 8 x 8 layer blocks below COMPRESS_TOL of their component's maximum dropped
    full_tensor_bytes = info_tensor_bytes(info)
    t0 = time.perf_counter()
    stored = plan.compress(COMPRESS_TOL)
    torch.cuda.synchronize()
    compress_s = time.perf_counter() - t0
    cinfo = plan.info
    crun = lambda: dm.demag_apply(plan.handle, m, Ms, H, stream, cinfo)  # noqa: E731
    for _ in range(max(args.warmup, 3)):
        crun()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    c_ms = max_over_ranks(float(time_steps(crun, args.steps, stream).mean()), dist, "cuda")
    cstage = np.mean([dm.demag_apply_timed(plan.handle, m, Ms, H, stream, cinfo) for _ in range(nk)], axis=0)
    H_cmp = H[0, SAMPLE_TARGET].clone()
    c_bytes = stored + (sbytes[2] - tensor)  # the contraction's bytes with the compressed tensor
    compressed = {
        "tol": COMPRESS_TOL, "stored_tensor_bytes": stored, "full_tensor_bytes": full_tensor_bytes,
        "stored_fraction": stored / full_tensor_bytes, "compress_s": compress_s,
        "value": whole_job_value(world, B, c_ms), "unit": "evals/s", "ms_per_step": c_ms,
        "contraction_ms": float(cstage[4]),
        "contraction_hbm": {"algorithmic_bytes": c_bytes, "achieved": c_bytes / (float(cstage[4]) * 1e-3) / 1e9,
                            "frac": c_bytes / (float(cstage[4]) * 1e-3) / 1e9 / peak, "unit": "GB/s"},
        "rel_l2_vs_uncompressed": float(torch.linalg.vector_norm((H[0, SAMPLE_TARGET] - H_gpu[0, SAMPLE_TARGET])
                                                                 .double()) /
                                        torch.linalg.vector_norm(H_gpu[0, SAMPLE_TARGET].double())),
        "note": "same plan after demag_plan_compress; the kept blocks are read and multiplied, dropped ones "
                "count as zero"}
    plan.close()
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": T, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 FFTs, 3xBF16 contraction with f32 accumulate", "data": "synthetic",
        "config": headline_config(c, th, desc, world, info),
        "gcell_layers_per_s": nx * ny * L * value / 1e9,
        "hbm_frac_min_bytes": ((2 * field + tensor) / (T * 1e-3) / 1e9) / peak,
        "kernels_ms": dict(zip(names, kernels_ms)),
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak,
                     "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback", "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(names[dom]),
                     "algorithmic_bytes": sbytes[dom]},
        "contraction_tensor_pipe": {"kernel": names[2], "useful_tflops": flops / (kernels_ms[2] * 1e-3) / 1e12,
                                    "issued_tflops_3_passes": 3 * flops / (kernels_ms[2] * 1e-3) / 1e12,
                                    "peak_bf16_tflops": bf16_peak,
                                    "frac": 3 * flops / (kernels_ms[2] * 1e-3) / 1e12 / bf16_peak,
                                    "note": "three BF16 passes against the measured sustained bf16 peak"},
        "e2e": {"value": whole_job_value(world, B, e2e_s * 1e3), "unit": "evals/s",
                "h2d_bytes_per_step": field, "d2h_bytes_per_step": field,
                "how": "demag_apply_host_async on page-locked buffers, %d consecutive steps (each copies its "
                       "16 states in and 16 fields out, the copies of one step overlapping the kernels of "
                       "the next), then demag_apply_host_wait" % ne,
                "one_call_at_a_time": {"value": whole_job_value(world, B, sync_s * 1e3), "unit": "evals/s",
                                       "how": "demag_apply_host, synchronised every step (%d steps)" % ns},
                "field_equals_device_run": e2e_match},
        "gpu_launches": 5 * args.steps,
        "plan_create_s": plan_s,
        "wall_s_timed_loop": wall,
        "compressed_tensor": compressed,
    }
    return line, m_np, H_gpu, H_cmp


def run_ours(args):
    import numpy as np
    import torch

    from paper_1910_07054_gb300 import inputs

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    peaks = load_peaks()
    clocks = ClockSampler(local)
    clocks.start()
    line, m_np, H_gpu, H_cmp = headline_measurement(args, world, rank, dist, peaks)
    line["clocks"] = clocks.stop()

    extras = {}
    if not args.no_extras:
        extras["mram256"] = mram_block(args, world, rank, dist, peaks, with_oracle=not args.no_cpu)
        if world == 1:
            extras["split_variants"] = batched_measurement(3, peaks, paths=(6, 7, 4, 3))
            extras["gradient"] = gradient_measurement(with_oracle=not args.no_parity)
            extras["nz_sweep"] = nz_sweep()
            extras["hysteresis"] = hysteresis_measurement()
            extras["surrogate"] = surrogate_measurement()
    if rank == 0:
        c, th, _ = headline_workload()
        L = len(th)
        need_pk = (not args.no_parity) or (world == 1 and not args.no_cpu)
        pk = headline_pair_kernels(c, th) if need_pk else None
        if not args.no_parity or (world == 1 and not args.no_cpu):
            t_s, H_ref = headline_oracle_sample(pk, m_np[0], inputs.MS_DEFAULT)
            H_s = H_gpu[0, SAMPLE_TARGET].double().cpu().numpy()
            line["rel_l2_vs_oracle"] = float(np.linalg.norm(H_s - H_ref) / np.linalg.norm(H_ref))
            line["rel_l2_sample"] = "target layer %d of state 0 against the float64 oracle (Eq. FFT_v2 pair by " \
                                    "pair)" % SAMPLE_TARGET
            H_c = H_cmp.double().cpu().numpy()
            line["compressed_tensor"]["rel_l2_vs_oracle"] = float(np.linalg.norm(H_c - H_ref) /
                                                                  np.linalg.norm(H_ref))
            if world == 1 and not args.no_cpu:
                line["cpu_baseline"] = {
                    "value": 1.0 / (L * t_s), "unit": "evals/s", "cores": 1, "kind": "oracle",
                    "sample": "one target layer (%d) of one state: oracle float64 hybrid_targets (numpy FFT, "
                              "single thread) over the 64 source layers in %.1f s; evals/s = 1 / (64 x sample); "
                              "pair kernels of the target row evaluated beforehand, not timed" % (SAMPLE_TARGET, t_s)}
                if not args.no_allcore:
                    line["cpu_baseline_all_cores"] = headline_oracle_allcore(pk, m_np, inputs.MS_DEFAULT, L)
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def gradient_measurement(steps=20, with_oracle=True):
    """The differentiation workload (256 x 256 cells of 2 nm, 10 layers with
    t ~ U[0.7, 4] nm, seed 0, one random state): the adjoint apply A^T gH
    (dH/dM) and d<H_z of layer 4>/d(thickness of layer 4), float plan.  The
    first thickness gradient builds the double-precision derivative tensor
    (all L^2 pairs); later ones reuse it (one apply of that tensor and a dot)."""
    import numpy as np
    import torch

    import paper_1910_07054_gb300 as dm
    from paper_1910_07054_gb300 import inputs
    c = inputs.CONFIGS["grad256"]
    th = [float(t) for t in inputs.thicknesses("grad256")]
    nx, ny, L, layer = c["nx"], c["ny"], len(th), 3
    plan = dm.Plan(nx, ny, c["dx"], c["dy"], th, precision=dm.PREC_FP32)
    info = plan.info
    m_np = inputs.random_unit_vectors((1, L, ny, nx), seed=0)
    m = torch.tensor(m_np, dtype=torch.float32, device="cuda")
    gH = torch.zeros_like(m)
    gH[0, layer, 2] = 1.0 / (nx * ny)
    gm = torch.empty_like(m)
    for _ in range(3):
        dm.demag_apply_adjoint(plan.handle, gH, inputs.MS_DEFAULT, gm, info=info)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        dm.demag_apply_adjoint(plan.handle, gH, inputs.MS_DEFAULT, gm, info=info)
    e1.record()
    torch.cuda.synchronize()
    adj_ms = e0.elapsed_time(e1) / steps
    t0 = time.perf_counter()
    g = dm.demag_thickness_grad(plan.handle, m, gH, inputs.MS_DEFAULT, layer, info=info)
    first_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for _ in range(steps):
        g = dm.demag_thickness_grad(plan.handle, m, gH, inputs.MS_DEFAULT, layer, info=info)
    again_ms = (time.perf_counter() - t0) / steps * 1e3
    plan.close()
    ref = None
    if with_oracle:
        # central difference (step 1e-4 nm) of the oracle's float64 mean H_z of
        # the layer, Eq. FFT_v2 for that target layer only
        from oracle import demag as odm
        from oracle import newell as onw
        h, vals = 1e-4, []
        for sgn in (1.0, -1.0):
            t = np.array(th)
            t[layer] += sgn * h
            pk = lambda i, j, t=t: onw.pair_kernel(nx, ny, c["dx"], c["dy"], t, i, j)  # noqa: E731
            vals.append(float(odm.hybrid_targets(pk, m_np[0], inputs.MS_DEFAULT, [layer])[layer][2].mean()))
        ref = (vals[0] - vals[1]) / (2 * h)
    return {"workload": "256x256 cells of 2x2 nm, 10 layers (t ~ U[0.7, 4] nm, seed 0), 1 random state, "
                        "float plan; d<H_z of layer 4>/dt_4 (1-based)",
            "adjoint_apply_ms": adj_ms, "adjoint_evals_per_s": 1e3 / adj_ms,
            "thickness_grad_first_s": first_s, "thickness_grad_cached_ms": again_ms,
            "dhz_dt": float(g), "dhz_dt_oracle_central_difference": ref,
            "dhz_dt_rel_err": None if ref is None else abs(float(g) - ref) / abs(ref)}


def nz_sweep(steps=20, n=256, nzs=(1, 2, 4, 8, 12, 16, 24, 32, 48, 64)):
    """The scaling sweep of Sec. 3.2 on GB300: n x n cells of 2 x 2 nm, nz layers
    of 1 nm (one thickness, so that both methods apply), one random state per
    evaluation, float plans: the hybrid of Eq. FFT_v2 (its default path for the
    stack) and the equidistant 3D FFT of Eq. FFT_3D.  Device time per
    evaluation (CUDA events, a 256 MB buffer written before each); fits of
    t = a nz^2 + b nz + c (hybrid) and t = a nz log2(nz) + b nz + c (3D FFT,
    the linear term for the nz-proportional FFTs in x and y), and the nz where
    the 3D FFT becomes the faster."""
    import numpy as np
    import torch

    import paper_1910_07054_gb300 as dm
    from paper_1910_07054_gb300 import inputs
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    rows = []
    for nz in nzs:
        m = torch.tensor(inputs.random_unit_vectors((1, nz, n, n), seed=nz), dtype=torch.float32, device="cuda")
        H = torch.empty_like(m)
        res = {"nz": nz}
        for name, make in (("hybrid", lambda: dm.Plan(n, n, 2.0, 2.0, (1.0,) * nz, precision=dm.PREC_FP32)),
                           ("fft3d", lambda: dm.Plan.equidistant(n, n, nz, 2.0, 2.0, 1.0, precision=dm.PREC_FP32))):
            t0 = time.perf_counter()
            plan = make()
            res[name + "_plan_s"] = time.perf_counter() - t0
            info = plan.info
            for k in range(3):
                flush.fill_(float(k))
                dm.demag_apply(plan.handle, m, 1.0, H, stream, info)
            ms = time_steps(lambda: dm.demag_apply(plan.handle, m, 1.0, H, stream, info), steps, stream,
                            before=lambda k: flush.fill_(float(k)))
            res[name + "_ms"] = float(np.median(ms))
            res[name + "_path"] = info["path"]
            if name == "hybrid":
                Hh = H.clone()
            else:
                res["rel_l2_fft3d_vs_hybrid"] = float(torch.linalg.vector_norm((H - Hh).double()) /
                                                      torch.linalg.vector_norm(Hh.double()))
            plan.close()
        rows.append(res)
    z = np.array([r["nz"] for r in rows], dtype=float)
    th = np.array([r["hybrid_ms"] for r in rows])
    t3 = np.array([r["fft3d_ms"] for r in rows])
    ch = np.linalg.lstsq(np.stack([z * z, z, np.ones_like(z)], 1), th, rcond=None)[0]
    c3 = np.linalg.lstsq(np.stack([z * np.log2(np.maximum(z, 1)), z, np.ones_like(z)], 1), t3, rcond=None)[0]
    grid = np.arange(1, 257)
    fh = ch[0] * grid ** 2 + ch[1] * grid + ch[2]
    f3 = c3[0] * grid * np.log2(grid) + c3[1] * grid + c3[2]
    cross_fit = next((int(g) for g, a, b in zip(grid, fh, f3) if b < a and g >= 2), None)
    cross_meas = next((r["nz"] for r in rows if r["fft3d_ms"] < r["hybrid_ms"]), None)
    return {"workload": "%dx%d cells of 2x2 nm, nz layers of 1 nm, 1 random state, float32 plans; device time "
                        "per evaluation (median of %d, cold L2)" % (n, n, steps),
            "rows": rows,
            "fit_hybrid_ms": {"a_nz2": ch[0], "b_nz": ch[1], "c": ch[2]},
            "fit_fft3d_ms": {"a_nzlog2nz": c3[0], "b_nz": c3[1], "c": c3[2]},
            "crossover_nz_measured": cross_meas, "crossover_nz_fit": cross_fit}


def hysteresis_measurement(steps=2000, b_max=2.5):
    """Sec. 4 switching simulation: the MRAM stack (64 x 64 cells over the 60 nm
    disk, layers [5, 1, 3.44, 1, 3] nm, the SAFM layers pinned +z / -z), CoFe free
    layer (Js = 1.75 T, A = 1.5e-11 J/m, Ku = 2.09e6 J/m^3 along z) relaxed by
    L-BFGS at each of `steps` field values from +b_max to -b_max along z (float
    plan); the sweep stops a few steps after the free layer switched."""
    import numpy as np
    import torch

    import paper_1910_07054_gb300 as dm
    from paper_1910_07054_gb300 import micromag as pmm
    dx, th, m, mask, layer = pmm.mram_stack()
    plan = dm.Plan(64, 64, dx, dx, th, precision=dm.PREC_FP32)
    mt = torch.tensor(m, dtype=torch.float32, device="cuda")
    bs = pmm.field_steps(b_max, steps)
    t0 = time.perf_counter()
    loop = pmm.hysteresis(plan, mt, layer, mask, bs, tol_torque=1e-4, stop_after_switch=5)
    wall = time.perf_counter() - t0
    plan.close()
    b_sw = pmm.switching_field(loop)
    return {"workload": "Sec. 4 MRAM stack 64x64 cells over 60 nm, layers [5, 1, 3.44, 1, 3] nm, SAFM pinned, CoFe free "
                        "layer; %d field steps from +%g to -%g T along z (%.2f mT), L-BFGS relaxation (torque < 1e-4 T) "
                        "at each" % (steps, b_max, b_max, 2e3 * b_max / steps),
            "switching_field_T": b_sw, "paper_switching_field_T": 1.51,
            "field_steps_run": len(loop), "relaxation_iterations": int(sum(x[2] for x in loop)),
            "wall_s": wall, "mz_at_zero_field": float(np.interp(0.0, [x[0] for x in loop][::-1],
                                                                [x[1] for x in loop][::-1]))}


def surrogate_measurement():
    """Sec. 4-like optimisation on the 256 x 256 x 8 stack: 2000 solver samples
    (layer 5 in [0.5, 5] nm, the others +-10%), network training, and Newton on
    the layer-5 thickness from 5 nm, exact vs surrogate-proposed steps."""
    import numpy as np

    from paper_1910_07054_gb300 import inputs
    from paper_1910_07054_gb300 import surrogate as sg
    solver = sg.ExactSolver(256, 2.0)
    t0 = time.perf_counter()
    T, Y = sg.generate_samples(solver, inputs.opt_samples(2000, seed=0))
    gen_s = time.perf_counter() - t0
    net = sg.Surrogate(seed=0)
    t0 = time.perf_counter()
    hist = net.fit(T[:1800], Y[:1800], steps=4000, lr=3e-3)
    fit_s = time.perf_counter() - t0
    held = net.predict(T[1800:])[:, 2]
    rmse = float(np.sqrt(np.mean((held - Y[1800:, 2]) ** 2)))
    start = inputs.OPT_BASE.copy()
    solver.solves = 0
    ex = sg.newton_exact(solver, start, tol=1e-6)
    solver.solves = 0
    su = sg.newton_surrogate(solver, net, start, tol=1e-6)
    t_star = ex[-1][0]
    n_ex = next(h[2] for h in ex if abs(h[0] - t_star) < 1e-3)
    n_su = next(h[2] for h in su if abs(h[0] - t_star) < 1e-3)
    return {"samples": 2000, "sample_generation_s": gen_s, "train_s": fit_s, "final_loss": hist[-1][1],
            "heldout_rmse_hz_over_ms": rmse, "t_opt_nm": t_star,
            "exact_solves_to_1e-3nm": {"newton_exact_adjoint": n_ex, "surrogate_proposed": n_su},
            "surrogate_final_t_nm": su[-1][0]}


def main():
    args = parse_args()
    if args.batched_only:
        paths = tuple(int(x) for x in args.batched_paths.split(","))
        print(json.dumps(batched_measurement(max(args.steps, 1), load_peaks(), args.batched_n, args.batched_layers,
                                             paths)), flush=True)
        return
    if args.grad_only:
        print(json.dumps(gradient_measurement(with_oracle=not args.no_parity)), flush=True)
        return
    if args.hysteresis_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(hysteresis_measurement()), flush=True)
        return
    if args.sweep_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(nz_sweep(max(args.steps, 5))), flush=True)
        return
    if args.mram_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(mram_block(args, 1, 0, None, load_peaks(), with_oracle=not args.no_cpu)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
