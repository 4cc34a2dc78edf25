#!/usr/bin/env python
"""Throughput benchmark of the BDIS hot path on GB300.

Default workload: one 640x480 surgical-like stereo pair (generator G2), 12x12
patches at stride 6, 4 pyramid levels, 8 Gauss-Newton iterations, variance
(PDF) estimate on, FP32 pyramids.  One step = one full coarse-to-fine pass
(pyramid, search, sigma_r, posterior + PDF, densify at every level) through
the C ABI.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 is launched with torch.distributed.run; every rank processes its own
independent pair (seed = rank), so the work shards with no collective in the
data path (weak scaling); only the timing uses a barrier and a max-reduce.
The reference arm (--impl reference) is the FP64 CPU oracle timed on the host
cores on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dense-disparity Mpix/s (fps @640x480) fwd and fwd+bwd, batched vs plain, at oracle match"
UNIT = "Mpix/s"
WORKLOAD = dict(workload="plain_640x480_var", generator="G2 surgical-like (seed = rank)",
                w=640, h=480, patch=12, stride=6, levels=4, iters=8, variance=1, storage="f32")
PARAMS = dict(patch=12, stride=6, levels=4, iters=8, variance=1, storage="f32")
BATCH_PARAMS = dict(patch=8, stride=4, levels=3, iters=8, variance=0, storage="f16")
L2_FLUSH_BYTES = 256 << 20   # larger than the 129 MB L2


def bench_config(ws):
    """The workload both arms measure (the reference arm prints the same)."""
    return dict(WORKLOAD, parallelism=f"replicas x{ws} (one pair per rank)",
                l2="flushed between timed steps (256 MiB write, outside the events)")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate_value(ws, units_per_rank, steps, max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (Mpix/s when units are pixels)."""
    return ws * units_per_rank * steps / (max_ms / 1e3) / 1e6


def rank_seed(rank, i=0, per_rank=1):
    """Each rank works on its own independent pairs: seed = per_rank*rank + i."""
    return per_rank * rank + i


def max_over_ranks(v, ws, device=None):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.index = str(device)
        try:
            import torch
            u = str(torch.cuda.get_device_properties(device).uuid)
            self.index = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.p is not None:
            time.sleep(0.2)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        loaded = [r for r in rows if r[4].isdigit() and int(r[4]) > 0] or rows
        sm = [float(r[1]) for r in loaded if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(loaded)}


# ---------------------------------------------------------------- roofline bookkeeping

def level_geometry(w, h, P, S, L):
    out = []
    for l in range(L):
        wl, hl = w, h
        for _ in range(l):
            wl, hl = (wl + 1) // 2, (hl + 1) // 2
        nx = (wl - P) // S + 1 + (1 if (wl - P) % S else 0)
        ny = (hl - P) // S + 1 + (1 if (hl - P) % S else 0)
        out.append((wl, hl, nx * ny))
    return out


def algorithmic_bytes(kernel, w, h, prm):
    if kernel == "persistent":   # every stage in one launch
        return sum(algorithmic_bytes(k, w, h, prm) for k in ("pyramid", "search", "fuse"))
    return _stage_bytes(kernel, w, h, prm)


def fwd_bwd_bytes(w, h, prm):
    """Algorithmic bytes of one differentiable step of one pair: the forward
    (float level-0 images) plus the loss and the finest-level adjoint.  Per
    level-0 pixel: loss reads L, R, D, valid (13 B) and writes dL/dD, dL/dI_l,
    dL/dI_r (12 B); the adjoint reads dL/dD, the weight sums, L, R and the
    gradient image (20 B) and accumulates into dL/dI_l, dL/dI_r (read + write,
    16 B).  Per level-0 patch: patch record 64 B, fusion record 16 B, dL/dd_k
    4 B."""
    P, S = prm["patch"], prm["stride"]
    fwd = sum(_stage_bytes(k, w, h, prm, level0_bytes=4) for k in ("pyramid", "search", "fuse"))
    npch = level_geometry(w, h, P, S, 1)[0][2]
    return fwd + w * h * (13 + 12 + 20 + 16) + npch * (64 + 16 + 4)


def _stage_bytes(kernel, w, h, prm, level0_bytes=1):
    """Bytes one pass of `kernel` over all levels must move (per pair).
    Image element sizes: level 0 u8 (float in the differentiable form),
    levels >= 1 and gradients the storage type; patch record 64 B; fusion
    record 16 B; fused maps 8 B/px."""
    P, S, L = prm["patch"], prm["stride"], prm["levels"]
    b = 2 if prm["storage"] == "f16" else 4
    geo = level_geometry(w, h, P, S, L)
    tot = 0
    for l, (wl, hl, npch) in enumerate(geo):
        img = level0_bytes if l == 0 else b
        px = wl * hl
        if kernel == "pyramid":
            nxt = geo[l + 1][0] * geo[l + 1][1] if l + 1 < L else 0
            tot += 2 * img * px + b * px + 2 * b * nxt     # read L, R; write G, next L, R
        elif kernel == "search":
            coarse = 4 * geo[l + 1][0] * geo[l + 1][1] if l + 1 < L else 0
            tot += 2 * img * px + b * px + coarse + 64 * npch  # read L, R, G, coarse D; write records
        elif kernel == "fuse":
            # read records, update posterior fields, write fusion records;
            # coarse D and Q; write D, Q (disp, var, valid at level 0)
            out = 9 if l == 0 else 8
            coarse = 8 * geo[l + 1][0] * geo[l + 1][1] if l + 1 < L else 0
            tot += 64 * npch + 16 * npch + 16 * npch + coarse + out * px
    return tot


def search_flops(w, h, prm):
    """Algorithmic FP32 operations of the patch search over all levels of one
    pair: per patch iters*P^2*6 (two taps, interpolation and the two
    accumulations of every GN step) + 5*P^2*5 (window samples, residual and
    energy sums) + 60 (setup); the PDF fit (about 400 per kept patch) runs
    in the fusion kernel and is not counted here."""
    P, S, L, it = prm["patch"], prm["stride"], prm["levels"], prm["iters"]
    per = it * P * P * 6 + 5 * P * P * 5 + 60
    return per * sum(n for _, _, n in level_geometry(w, h, P, S, L))


def alu_peak_tflops(sm_mhz=None):
    """FP32 FMA peak: 152 SMs x 128 lanes x 2 flops x SM clock (the maximum
    clock of MEASURED_PEAKS.json unless a measured median is given)."""
    pk = measured_peaks() or {}
    mhz = sm_mhz or pk.get("sm_max_mhz", 2070.0)
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


KERNEL_SOURCES = ("bdis_kernels.cu", "bdis_device.cuh", "bdis_internal.cuh")


def code_digest(texts):
    """Digest of CUDA sources without their comments and blank lines (what
    the compiler sees), so that a comment edit keeps a capture valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    for t in texts:
        t = re.sub(r"/\*.*?\*/", "", t, flags=re.S)
        t = re.sub(r"//[^\n]*", "", t)
        lines = [ln.rstrip() for ln in t.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def kernel_source_digest():
    return code_digest(open(os.path.join(ROOT, "paper_2205_03133_gb300", "csrc", f)).read()
                       for f in KERNEL_SOURCES)


def recorded_traffic(kernel):
    """DRAM bytes per step (sum over the step's launches) of `kernel` on this
    workload, from the committed ncu summary -- only if that capture was
    taken on the current kernel sources (digest match), else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_plain_640x480_var.md")
    try:
        kv = dict(line.split(":", 1) for line in open(path) if line.startswith(("source_digest:", "dram_bytes_per_step:")))
    except Exception:
        return None
    if kv.get("source_digest", "").strip() != kernel_source_digest():
        return None
    try:
        return int(float(kv["dram_bytes_per_step"]))
    except Exception:
        return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ---------------------------------------------------------------- CPU baseline (oracle)

def host_cpu():
    """Usable host cores and the CPU model string."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return cores, f"{model or 'unknown'} ({platform.machine()})"


def _oracle_worker(job):
    """One host process: the oracle on its own pair until the wall budget."""
    left, right, prm, budget = job
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    op = oracle.make_params(**prm)
    runs, t0 = 0, time.perf_counter()
    while True:
        oracle.match(op, left, right)
        runs += 1
        if time.perf_counter() - t0 >= budget:
            break
    return runs, time.perf_counter() - t0


def cpu_all_cores(prm, cores, budget_s=8.0):
    """The oracle on every host core at once, one independent 640x480 pair
    (G2, seed 100 + i) per process (the oracle itself is single-threaded),
    until the wall budget: total pixels over the slowest process's time."""
    import multiprocessing as mp

    import synth
    jobs = []
    for i in range(cores):
        pr = synth.g2_pair(640, 480, 100 + i)
        jobs.append((pr.left, pr.right, dict(prm), budget_s))
    ctx = mp.get_context("spawn")   # no fork after CUDA is initialised
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    runs = sum(r for r, _ in res)
    el = max(t for _, t in res)
    return {"value": round(runs * 640 * 480 / el / 1e6, 4), "unit": UNIT, "cores": cores,
            "sample": f"{runs} full 640x480 pairs over {cores} processes (one pair each, "
                      f"FP64 C oracle, 1 thread per process), {el:.1f} s wall"}


def cpu_baseline(pair, prm, budget_s=12.0, gpu_out=None, all_cores=True):
    """The FP64 C oracle as it stands, one thread, on full pairs of the
    workload until `budget_s` of CPU time is spent (at least one run); then
    the same oracle on every host core (one process per core)."""
    import numpy as np

    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    op = oracle.make_params(**{k: v for k, v in prm.items()})
    oracle.build()
    runs, t0 = 0, time.perf_counter()
    first = None
    while True:
        out = oracle.match(op, pair.left, pair.right, trace=gpu_out is not None and runs == 0)
        first = first or out
        runs += 1
        el = time.perf_counter() - t0
        if el >= budget_s or runs >= 200:
            break
    px = pair.left.size * runs
    cores, model = host_cpu()
    res = {"value": round(px / el / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{runs} full {pair.left.shape[1]}x{pair.left.shape[0]} pairs "
                     f"(all {prm['levels']} levels, variance on), FP64 C, 1 thread, {el:.1f} s",
           "host_cores": cores, "cpu_model": model}
    if all_cores and cores > 1:
        res["all_cores"] = cpu_all_cores(prm, cores)
    if gpu_out is not None:
        from parity import compare_outputs
        disp, var, valid, rec0, gp = gpu_out
        m = compare_outputs(gp, first, disp, var, valid, rec0)
        res["parity_vs_gpu"] = {k: (round(v, 8) if isinstance(v, float) else v) for k, v in m.items()}
    return res


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth
    pair = synth.config_pair("plain_640x480_var", seed=0)
    op = oracle.make_params(**PARAMS)
    oracle.build()
    t = time.perf_counter()
    oracle.match(op, pair.left, pair.right)
    t_full = time.perf_counter() - t
    # each step: a bounded sample of the workload (a full-width crop of the
    # pair) so that warm-up + timed steps stay near one minute in total
    budget = 60.0 / max(1, args.steps + args.warmup)
    hmin = 12 * 8 + 12
    hc = 480 if t_full <= budget else max(hmin, int(480 * budget / t_full) // 8 * 8)
    L, R = pair.left[:hc].copy(), pair.right[:hc].copy()
    for _ in range(max(0, args.warmup - 1)):
        oracle.match(op, L, R)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.match(op, L, R)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    px = L.size * args.steps
    val = px / tot / 1e6
    cores, model = host_cpu()
    sample = (f"each step a 640x{hc} crop of the 640x480 pair (full coarse-to-fine, variance on); "
              f"FP64 C oracle, 1 thread of {cores} host cores ({model})")
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(ws),
            "cpu_baseline": {"value": round(val, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "crop_h": hc, "host_cores": cores,
                             "cpu_model": model},
            "e2e": {"value": round(val, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- ours

def relaunch_distributed(n):
    """`--gpus N` without a distributed environment: run this same command
    under torch.distributed.run, one rank per GPU on this node."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node",
           str(n), "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


L2_PEAK_SOURCE = ("measured in bench.py: bdis_probe_l2_read, one launch re-reading a 48 MiB "
                  "L2-resident buffer 40 times with 16-byte loads (best of 5)")


def l2_copy_gbs(dev, stream, mib=48, reps=40):
    """L2 read bandwidth: one launch of the library's probe re-reads a
    mib-MiB buffer (resident in the 129 MB L2 after a warm-up pass) `reps`
    times; bytes read over CUDA-event time, best of five."""
    import ctypes as C

    import torch

    from paper_2205_03133_gb300 import _binding as B
    a = torch.ones(mib << 18, dtype=torch.float32, device=dev)
    sh = C.c_void_p(stream.cuda_stream)
    nbytes = a.numel() * 4
    B.check(B.lib().bdis_probe_l2_read(C.c_void_p(a.data_ptr()), nbytes, 2, sh))
    best = float("inf")
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.check(B.lib().bdis_probe_l2_read(C.c_void_p(a.data_ptr()), nbytes, reps, sh))
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return nbytes * reps / (best / 1e3) / 1e9


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only", default="all", choices=["all", "batched", "fwdbwd"],
                    help="batched / fwdbwd: only the 64-pair batched form / the differentiable "
                         "form (used for profiling)")
    ap.add_argument("--form", default="auto", choices=["auto", "launches", "persistent"],
                    help="execution form of the plain workload (auto: the autotuner's choice)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return relaunch_distributed(args.gpus)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_2205_03133_gb300 as bd
    import synth
    from paper_2205_03133_gb300 import build as _build
    _build.build()

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    init_dist(ws, "nccl")
    dev = torch.device("cuda", local)
    B = bd.B
    if args.only == "batched":
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        stream = torch.cuda.Stream(device=dev)
        res = bench_batched(bd, dev, stream, flush, rank, ws, steps=args.steps,
                            warmup=args.warmup, compare_plain=False, form=args.form)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "batched": res}))
        return 0
    if args.only == "fwdbwd":
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        stream = torch.cuda.Stream(device=dev)
        res = bench_fwd_bwd(bd, dev, stream, flush, rank, ws, steps=args.steps, warmup=args.warmup)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "fwd_bwd": res}))
        return 0

    pair = synth.config_pair("plain_640x480_var", seed=rank_seed(rank))
    h, w = pair.left.shape
    Ld = torch.from_numpy(pair.left).to(dev)
    Rd = torch.from_numpy(pair.right).to(dev)
    out = (torch.empty((h, w), dtype=torch.float32, device=dev),
           torch.empty((h, w), dtype=torch.float32, device=dev),
           torch.empty((h, w), dtype=torch.uint8, device=dev))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    m = bd.BDIS(**PARAMS)
    if args.form != "auto":
        m.set_option(B.OPT_FORM, {"launches": 1, "persistent": 2}[args.form])
    launches_per_step = None  # counted by the profiling pass below

    def step():
        m.match(Ld, Rd, out=out, stream=stream)

    clocks = ClockSampler(local)
    clocks.start()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step()
    torch.cuda.synchronize()

    # ---- timed: device time of exactly K steps, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    clocks.mark("t0")
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks.mark("t1")
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    dev_ms_max = max_over_ranks(dev_ms, ws, dev)
    value = aggregate_value(ws, w * h, args.steps, dev_ms_max)

    # ---- per-kernel event times (profiling pass, plain launches)
    B.lib().bdis_set_option(m._h, B.OPT_PROFILE, 1)
    prof = B.bdis_profile()
    B.lib().bdis_get_profile(m._h, prof, 1)
    n_prof = max(20, min(args.steps, 200))
    with torch.cuda.stream(stream):
        for _ in range(n_prof):
            flush.zero_()
            step()
    torch.cuda.synchronize()
    B.check(B.lib().bdis_get_profile(m._h, prof, 1), m._h)
    B.lib().bdis_set_option(m._h, B.OPT_PROFILE, 0)
    kernels = {}
    for i, name in enumerate(B.KERNEL_NAMES[:len(prof.launches)]):
        if prof.launches[i]:
            kernels[name] = {"launches_per_step": prof.launches[i] // n_prof,
                             "ms_per_step": prof.ms[i] / n_prof,
                             "avg_launch_us": prof.ms[i] / prof.launches[i] * 1e3,
                             "us_per_launch_by_level": {
                                 str(l): round(prof.ms_level[i][l] / prof.launches_level[i][l] * 1e3, 3)
                                 for l in range(8) if prof.launches_level[i][l]}}
    launches_per_step = sum(k["launches_per_step"] for k in kernels.values())
    tot_k = sum(k["ms_per_step"] for k in kernels.values())
    for k in kernels.values():
        k["share"] = round(k["ms_per_step"] / tot_k, 4)
        k["ms_per_step"] = round(k["ms_per_step"], 5)
        k["avg_launch_us"] = round(k["avg_launch_us"], 3)
    st = m.stats(stream)
    form = {1: "persistent (every stage in one cooperative launch)",
            2: "coarse levels in one cooperative launch, finer levels as a launch sequence "
               "(CUDA graph, programmatic dependent launch)"}.get(
        st["persistent"], "launch sequence (CUDA graph, programmatic dependent launch)")
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    per_step_bytes = algorithmic_bytes(dom, w, h, PARAMS)
    achieved = per_step_bytes / (kernels[dom]["ms_per_step"] / 1e3) / 1e9
    l2_peak = l2_copy_gbs(dev, stream)
    roofline = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 2),
                "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 5),
                "traffic": recorded_traffic(dom),
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback",
                "algorithmic_bytes_per_step": per_step_bytes,
                "launches_per_step": kernels[dom]["launches_per_step"],
                "time_source": "CUDA events around each launch of the kernel (profiling pass of "
                               "the same calls: plain launches, no graph)",
                "l2": {"achieved": round(achieved, 2), "peak": round(l2_peak, 1), "unit": "GB/s",
                       "frac": round(achieved / l2_peak, 5),
                       "peak_source": L2_PEAK_SOURCE}}
    roofline_alu = None
    if "search" in kernels:
        fl = search_flops(w, h, PARAMS)
        ach = fl / (kernels["search"]["ms_per_step"] / 1e3) / 1e12
        pk = alu_peak_tflops()
        roofline_alu = {"kernel": "search", "bound": "alu", "achieved": round(ach, 4),
                        "peak": round(pk, 2), "unit": "TFLOP/s", "frac": round(ach / pk, 5),
                        "algorithmic_flops_per_step": fl,
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}

    # ---- end to end through the host-buffer entry point (pinned buffers)
    hL = torch.from_numpy(pair.left).pin_memory()
    hR = torch.from_numpy(pair.right).pin_memory()
    hD = torch.empty((h, w), dtype=torch.float32).pin_memory()
    hV = torch.empty((h, w), dtype=torch.float32).pin_memory()
    hM = torch.empty((h, w), dtype=torch.uint8).pin_memory()
    sh = B.C.c_void_p(stream.cuda_stream)
    e2e_steps = max(10, min(args.steps, 200))

    def hstep():
        m.match_host_ptr(hL.data_ptr(), hR.data_ptr(), w, h, hD.data_ptr(), hV.data_ptr(),
                         hM.data_ptr(), sh)

    with torch.cuda.stream(stream):
        for _ in range(3):
            flush.zero_()
            hstep()
    torch.cuda.synchronize()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(e2e_steps)]
    with torch.cuda.stream(stream):
        for k in range(e2e_steps):
            flush.zero_()
            ev2[k][0].record(stream)
            hstep()
            ev2[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev2), ws, dev)
    # the same with staging copies through device memory (cudaMemcpyAsync)
    B.check(B.lib().bdis_set_option(m._h, B.OPT_HOST_MAPPED, 0), m._h)
    with torch.cuda.stream(stream):
        for _ in range(3):
            flush.zero_()
            hstep()
    torch.cuda.synchronize()
    ev3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(e2e_steps)]
    with torch.cuda.stream(stream):
        for k in range(e2e_steps):
            flush.zero_()
            ev3[k][0].record(stream)
            hstep()
            ev3[k][1].record(stream)
    torch.cuda.synchronize()
    B.check(B.lib().bdis_set_option(m._h, B.OPT_HOST_MAPPED, 1), m._h)
    staged_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev3), ws, dev)
    e2e = {"value": round(ws * w * h * e2e_steps / (e2e_ms / 1e3) / 1e6, 3), "unit": UNIT,
           "h2d_bytes_per_step": 2 * w * h, "d2h_bytes_per_step": (4 + 4 + 1) * w * h,
           "steps": e2e_steps,
           "api": "bdis_match_host with pinned host buffers, read and written in place by the "
                  "kernels over the host link (no staging copies)",
           "staged_copies_value": round(ws * w * h * e2e_steps / (staged_ms / 1e3) / 1e6, 3)}
    clock_info = clocks.stop()

    # ---- batched form: 64 uneven pairs, one launch per stage per level
    batched = None
    fwd_bwd = None
    modes = None
    depth_line = None
    coverage = None
    if not args.no_batched:
        batched = bench_batched(bd, dev, stream, flush, rank, ws, form=args.form)
        fwd_bwd = bench_fwd_bwd(bd, dev, stream, flush, rank, ws)
        modes = bench_modes(bd, dev, stream, flush, ws, Ld, Rd, out, w, h)
        coverage = variance_coverage_experiment(bd, dev, stream)
        depth_line = bench_depth(bd, dev, stream, flush, ws)

    result = None
    if rank == 0:
        cpu = None
        if not args.no_cpu:
            rec0 = None
            with torch.cuda.stream(stream):
                step()
            torch.cuda.synchronize()
            rec0 = m.level_view(0, 0)["patches"]
            gpu_out = (out[0].cpu().numpy(), out[1].cpu().numpy(), out[2].cpu().numpy(), rec0,
                       m.params)
            cpu = cpu_baseline(pair, PARAMS, gpu_out=gpu_out)
        result = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dev_ms_max / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "fps": round(value / (w * h / 1e6), 2),
            "config": bench_config(ws),
            "gpu_launches": launches_per_step * args.steps,
            "form": form,
            "kernels": kernels,
            "roofline": roofline,
            "roofline_alu": roofline_alu,
            "e2e": e2e,
            "clocks": clock_info,
            "cpu_baseline": cpu,
            "batched": batched,
            "fwd_bwd": fwd_bwd,
            "modes": modes,
            "variance_coverage": coverage,
            "depth": depth_line,
            "paper_context": "BDIS(VAR) 0.072 s per 640x480 frame (4.27 Mpix/s) on one i5-9400 "
                             "core, finest scale 2^1 (Table VIII); 17 Hz claim (abstract)",
        }
        print(json.dumps(result))
    m.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


DIFF_PARAMS = dict(patch=8, stride=4, levels=3, iters=8, variance=0, storage="f32")


def bench_fwd_bwd(bd, dev, stream, flush, rank, ws, steps=10, warmup=3):
    """Differentiable form: 16 float pairs of 640x480 (G1, seeds 16*rank + i),
    one step = batched forward + L1 reprojection / smoothness loss + adjoint
    (gradients w.r.t. both images and the patch disparities)."""
    import torch

    import synth
    n, w, h = 16, 640, 480
    Ls, Rs = [], []
    for i in range(n):
        p = synth.g1_pair(w, h, rank_seed(rank, i, 16))
        Ls.append(torch.from_numpy(p.left.astype("float32")).to(dev))
        Rs.append(torch.from_numpy(p.right.astype("float32")).to(dev))
    m = bd.BDIS(**DIFF_PARAMS)
    B = bd.B
    outs = [(torch.empty((h, w), device=dev), None, torch.empty((h, w), dtype=torch.uint8, device=dev))
            for _ in range(n)]

    def fwd():
        m.match_f32(Ls, Rs, outs=outs, stream=stream)

    bufs = None

    def fwd_bwd():
        nonlocal bufs
        fwd()
        if bufs is None:
            bufs = m.loss_and_grad(0.1, stream=stream)
            return
        arr = bd._grad_table(m, bufs)
        st = B.C.c_void_p(stream.cuda_stream)
        B.check(B.lib().bdis_loss(m._h, None, B.C.c_float(0.1), arr, st), m._h)
        B.check(B.lib().bdis_backward(m._h, None, arr, st), m._h)

    def run(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(k)]
        with torch.cuda.stream(stream):
            for i in range(k):
                flush.zero_()
                ev[i][0].record(stream)
                fn()
                ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / k

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fwd_bwd()
    torch.cuda.synchronize()
    t_fb = max_over_ranks(run(fwd_bwd, steps), ws, dev)
    t_f = max_over_ranks(run(fwd, steps), ws, dev)
    loss = float(torch.stack([b["loss"] for b in bufs]).mean().item())
    # the adjoint through every level (coarse levels through Eq. 10, pyramid)
    B.check(B.lib().bdis_set_option(m._h, B.OPT_ADJOINT_LEVELS, 1), m._h)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fwd_bwd()
    torch.cuda.synchronize()
    t_fb_all = max_over_ranks(run(fwd_bwd, steps), ws, dev)
    m.close()
    px = n * w * h
    by = n * fwd_bwd_bytes(w, h, DIFF_PARAMS)
    pk = measured_peaks() or {}
    hbm = pk.get("hbm_gbs", 6800.0)
    l2 = l2_copy_gbs(dev, stream)
    ach = by / (t_fb / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(ach / hbm, 4), "algorithmic_bytes_per_step": by,
            "l2": {"achieved": round(ach, 1), "peak": round(l2, 1), "unit": "GB/s",
                   "frac": round(ach / l2, 4), "peak_source": L2_PEAK_SOURCE},
            "scope": "whole fwd+bwd step (all its kernels): forward algorithmic bytes with float "
                     "level-0 images plus the loss and finest-level adjoint bytes "
                     "(bench.py fwd_bwd_bytes)"}
    return {"workload": "16 float pairs 640x480 (G1), P8 S4 L3, 8 iters, loss = L1 reprojection "
                        "+ 0.1 smoothness; grads w.r.t. both images and patch disparities",
            "roofline": roof,
            "value": round(ws * px / (t_fb / 1e3) / 1e6, 2), "unit": UNIT,
            "ms_per_step": round(t_fb, 4), "fwd_only_value": round(ws * px / (t_f / 1e3) / 1e6, 2),
            "fwd_only_ms": round(t_f, 4), "mean_loss": round(loss, 5),
            "all_levels_value": round(ws * px / (t_fb_all / 1e3) / 1e6, 2),
            "all_levels_ms_per_step": round(t_fb_all, 4)}


def bench_batched(bd, dev, stream, flush, rank, ws, steps=10, warmup=3, compare_plain=True,
                  form="auto"):
    """64 pairs of uneven sizes (24x640x480, 16x960x540, 16x1280x720,
    8x1920x1080; G1 generator, seeds 64*rank + i) in one batched call per
    step, against 64 sequential plain calls."""
    import torch

    import synth
    sizes = synth.batch_sizes_uneven()
    Ls, Rs, outs = [], [], []
    for i, (w, h) in enumerate(sizes):
        p = synth.g1_pair(w, h, rank_seed(rank, i, 64))
        Ls.append(torch.from_numpy(p.left).to(dev))
        Rs.append(torch.from_numpy(p.right).to(dev))
        outs.append((torch.empty((h, w), dtype=torch.float32, device=dev), None,
                     torch.empty((h, w), dtype=torch.uint8, device=dev)))
    px = sum(w * h for w, h in sizes)
    m = bd.BDIS(**BATCH_PARAMS)
    mp = bd.BDIS(**BATCH_PARAMS)
    if form != "auto":
        m.set_option(bd.B.OPT_FORM, {"launches": 1, "persistent": 2}[form])

    def run(fn, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        with torch.cuda.stream(stream):
            for k in range(n):
                flush.zero_()
                ev[k][0].record(stream)
                fn()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / n

    batched_fn = lambda: m.match_batched(Ls, Rs, outs=outs, stream=stream)  # noqa: E731

    def plain_fn():
        for i in range(len(sizes)):
            mp.match(Ls[i], Rs[i], out=outs[i], stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            batched_fn()
            if compare_plain:
                plain_fn()
    torch.cuda.synchronize()
    t_b = max_over_ranks(run(batched_fn, steps), ws, dev)
    if not compare_plain:
        m.close()
        mp.close()
        return {"value": round(ws * px / (t_b / 1e3) / 1e6, 2), "unit": UNIT,
                "ms_per_batch": round(t_b, 4)}
    t_p = max_over_ranks(run(plain_fn, max(3, steps // 2)), ws, dev)
    bd.B.lib().bdis_set_option(m._h, bd.B.OPT_PROFILE, 1)
    prof = bd.B.bdis_profile()
    bd.B.lib().bdis_get_profile(m._h, prof, 1)
    with torch.cuda.stream(stream):
        for _ in range(3):
            flush.zero_()
            batched_fn()
    torch.cuda.synchronize()
    bd.B.lib().bdis_get_profile(m._h, prof, 1)
    kern = {n: round(prof.ms[i] / 3, 4) for i, n in enumerate(bd.B.KERNEL_NAMES) if prof.launches[i]}
    m.close()
    mp.close()
    roof = None
    if "search" in kern:
        fl = sum(search_flops(w, h, BATCH_PARAMS) for w, h in sizes)
        by = sum(algorithmic_bytes("search", w, h, BATCH_PARAMS) for w, h in sizes)
        t = kern["search"] / 1e3
        pk = measured_peaks() or {}
        hbm = pk.get("hbm_gbs", 6800.0)
        l2 = l2_copy_gbs(dev, stream)
        roof = {"kernel": "search",
                "alu": {"achieved": round(fl / t / 1e12, 3), "peak": round(alu_peak_tflops(), 2),
                        "unit": "TFLOP/s", "frac": round(fl / t / 1e12 / alu_peak_tflops(), 4)},
                "hbm": {"achieved": round(by / t / 1e9, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(by / t / 1e9 / hbm, 4)},
                "l2": {"achieved": round(by / t / 1e9, 1), "peak": round(l2, 1), "unit": "GB/s",
                       "frac": round(by / t / 1e9 / l2, 4),
                       "peak_source": L2_PEAK_SOURCE},
                "algorithmic_flops": fl, "algorithmic_bytes": by}
    return {"workload": "64 uneven pairs (24x640x480, 16x960x540, 16x1280x720, 8x1920x1080), "
                        "P8 S4 L3, 8 iters, fp16 pyramids",
            "value": round(ws * px / (t_b / 1e3) / 1e6, 2), "unit": UNIT,
            "ms_per_batch": round(t_b, 4),
            "plain_sequential_ms": round(t_p, 4),
            "plain_sequential_value": round(ws * px / (t_p / 1e3) / 1e6, 2),
            "speedup_vs_plain": round(t_p / t_b, 3), "kernel_ms_per_batch": kern,
            "roofline": roof}


MODES = {
    # the paper's parameter set (Sec. IV-A): scales 2^5 .. 2^1, patch 10,
    # overlap 0.55 (stride 4), 12 iterations, upsampled to full resolution
    "paper_preset": dict(patch=10, stride=4, levels=6, iters=12, finest_level=1, variance=1),
    "dis_weights": dict(PARAMS, weight_mode="dis"),
    "fast_exp": dict(PARAMS, fast_exp=1),
    "no_sgmm_no_c2f": dict(PARAMS, use_sgmm=0, use_c2f=0),
    "sigma_r_fixed_8": dict(PARAMS, sigma_r_mode="fixed"),
}


def bench_modes(bd, dev, stream, flush, ws, Ld, Rd, out, w, h, steps=200, warmup=5):
    """The plain 640x480 workload under the optional modes (same pair, same
    outputs), device time per call with L2 flushed between calls."""
    import torch
    res = {}
    for name, kw in MODES.items():
        m = bd.BDIS(**kw)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                flush.zero_()
                m.match(Ld, Rd, out=out, stream=stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.zero_()
                ev[k][0].record(stream)
                m.match(Ld, Rd, out=out, stream=stream)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / steps, ws, dev)
        st = m.stats(stream)
        res[name] = {"params": {k: v for k, v in kw.items()}, "ms_per_call": round(ms, 5),
                     "value": round(ws * w * h / (ms / 1e3) / 1e6, 2), "unit": UNIT,
                     "valid_pixels": int(st["valid_pixels"])}
        m.close()
    return res


def variance_coverage(disp, var, valid, gt, z=1.96):
    """Fraction of valid pixels whose error is within z standard deviations
    of the estimated variance (the synthetic analogue of Table VI)."""
    import numpy as np
    v = valid.astype(bool) & np.isfinite(var) & (var > 0)
    e = np.abs(disp[v].astype(np.float64) - gt[v])
    return {"valid_frac": round(float(valid.astype(bool).mean()), 4),
            "coverage": round(float((e <= z * np.sqrt(var[v])).mean()), 4) if v.any() else None,
            "mean_abs_err_px": round(float(e.mean()), 4) if v.any() else None,
            "median_abs_err_px": round(float(np.median(e)), 4) if v.any() else None,
            "median_sigma_px": round(float(np.median(np.sqrt(var[v]))), 4) if v.any() else None}


def variance_coverage_experiment(bd, dev, stream):
    """|e| <= 1.96 sigma on seeded G1 / G2 pairs with known ground truth, for
    the bench parameters and for the paper's parameter set (Sec. IV-A)."""
    import torch

    import synth
    res = {}
    cases = {
        "g1_640x480": (synth.g1_pair(640, 480, 0), dict(PARAMS)),
        "g2_640x480": (synth.g2_pair(640, 480, 0), dict(PARAMS)),
        "g1_640x480_paper_preset": (synth.g1_pair(640, 480, 0), dict(MODES["paper_preset"])),
        "g2_640x480_paper_preset": (synth.g2_pair(640, 480, 0), dict(MODES["paper_preset"])),
    }
    for name, (pr, kw) in cases.items():
        kw["variance"] = 1
        m = bd.BDIS(**kw)
        d, v, ok = m.match(torch.from_numpy(pr.left).to(dev), torch.from_numpy(pr.right).to(dev),
                           stream=stream)
        torch.cuda.synchronize()
        res[name] = variance_coverage(d.cpu().numpy(), v.cpu().numpy(), ok.cpu().numpy(), pr.gt_left())
        m.close()
    return res


def bench_depth(bd, dev, stream, flush, ws, frames=64, steps=20, warmup=3):
    """Depth and depth variance (Eq. 13, Eq. 17) of 64 full-HD disparity and
    variance maps: an HBM-bound elementwise kernel, 16 B per pixel."""
    import torch
    n = frames * 1920 * 1080
    g = torch.Generator(device=dev).manual_seed(0)
    d = torch.rand(n, device=dev, generator=g) * 100 + 1
    v = torch.rand(n, device=dev, generator=g)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            z, zv = bd.depth(d, v, fb=2.56, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            z, zv = bd.depth(d, v, fb=2.56, stream=stream)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / steps, ws, dev)
    by = 16 * n
    pk = measured_peaks() or {}
    hbm = pk.get("hbm_gbs", 6800.0)
    del d, v, z, zv
    torch.cuda.empty_cache()
    return {"workload": f"{frames} x 1920x1080 disparity + variance maps (f32)",
            "ms": round(ms, 4), "value": round(ws * n / (ms / 1e3) / 1e6, 1), "unit": "Mpix/s",
            "roofline": {"bound": "hbm", "achieved": round(by / (ms / 1e3) / 1e9, 1),
                         "peak": hbm, "unit": "GB/s", "frac": round(by / (ms / 1e3) / 1e9 / hbm, 4),
                         "algorithmic_bytes": by}}


if __name__ == "__main__":
    sys.exit(main())
