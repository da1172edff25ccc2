#!/usr/bin/env python
"""Throughput of the PS-quadrature hot path on one GB300 (or N independent replicas).

One step = one psq_compute of a whole job (grid + weights, STO and aux-potential evaluation,
contraction, reduction, assembly of every requested integral class) on synthetic inputs
resident in device memory.  Metric: useful point-basis^2 contractions per second (one
contraction = one w f g multiply-accumulate into one matrix element; the count follows the
assembly rule: every matrix element integrated once on one grid).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3h6]
                    [--precision fp64|mixed] [--impl psq|reference]

The default workload is the propanediyl-shaped C3H6 job (9 atoms, 228 basis / 693 aux
functions, 36 pair + 252 refined grids, 55.8 M points), the largest single-GPU configuration.
Prints ONE JSON line on rank 0, with the mixed path's largest absolute error per class
against the FP64 oracle on sampled blocks (and against the plain FP64 GPU path on every
element), the plain FP64 path's throughput on the same job, and a short serving run.
``--impl reference`` times the CPU oracle (the paper's method written plainly in numpy FP64)
on the host cores instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pt·basis² contractions/s vs plain FP64; serve p50/p99 latency at err≤1e-9"
UNIT = "contractions/s"
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate (no measured FP64 peak is provided)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: a few seconds of the workload)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="psq", choices=["psq", "reference"])
    ap.add_argument("--workload", default="c3h6")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="steps of the plain FP64 path timed beside")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the per-class errors against the oracle")
    ap.add_argument("--no-serve-block", action="store_true", help="skip the short serving run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default work split")
    ap.add_argument("--no-ri", action="store_true", help="skip timing the RI 4-index assembly")
    ap.add_argument("--serve", action="store_true", help="serving benchmark instead of the step benchmark")
    ap.add_argument("--scan", action="store_true", help="Fig. 6 displacement scans through the serving loop")
    ap.add_argument("--ri-sizes", default=None,
                    help="n,m: time the RI 4-index assembly alone on seeded synthetic (P|Q) (n x n) and (P|ij) "
                         "(n x m) matrices")
    ap.add_argument("--rates", default="10,20,50,100,200,500", help="serving: Poisson arrival rates (jobs/s)")
    ap.add_argument("--jobs", type=int, default=300, help="serving: jobs per rate")
    ap.add_argument("--serve-window", type=int, default=32,
                    help="serving: jobs submitted and unfinished at most (the rest queue on the host)")
    ap.add_argument("--baseline-jobs", type=int, default=6, help="serving: jobs timed on the per-job FP64 path")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate(times_s, units_per_rank, world, device="cuda"):
    """Replicas (weak scaling): every rank processed `units_per_rank` in its own wall times
    `times_s` (one per timed region); the job's time of a region is the slowest rank's, and its
    throughput all ranks' units over that time.  Returns (max times, throughputs)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor(list(times_s), dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        times_s = [float(x) for x in t.tolist()]
    return list(times_s), [world * u / t for u, t in zip(units_per_rank, times_s)]


# ------------------------------------------------------------------------------ CPU oracle

def oracle_sample(job):
    """The reference arm's step: a bounded sample of the workload for the CPU oracle, the
    sub-molecule of atoms 0 and 1 (their basis and aux shells, their pair's grid spec, every
    class), i.e. one pair grid."""
    import synth
    sub = synth.sub_molecule(job, (0, 1))
    spec = sub.specs[0]
    return sub, "atoms 0-1 of %s (one %dx%dx%d Q%d%d%d pair grid, %s classes)" % (
        job.name, spec[0], spec[1], spec[2], spec[3], spec[4], spec[5], "all" if job.mask == 31 else job.mask)


def baseline_sample(job):
    """The cpu_baseline sample: a three-atom sub-molecule of the workload (atoms 0, 1 and the
    last atom: for C3H6 two carbons and a hydrogen) with every class, i.e. three pair grids and
    three grids refined around the third centre, 3-centre V and (P|ij) included; the whole job
    when it has at most three atoms."""
    import synth
    if job.n_atoms <= 3:
        return job, "%s in full (%d grids, every class)" % (job.name, job.n_atoms * (job.n_atoms - 1) // 2 * (
            1 + (job.n_atoms - 2)))
    keep = (0, 1, job.n_atoms - 1)
    sub = synth.sub_molecule(job, keep)
    return sub, "atoms %d, %d, %d of %s (3 pair + 3 refined grids with its grid specs, every class)" % (
        keep + (job.name,))


def time_oracle(job, min_seconds=10.0, max_runs=20):
    import oracle
    sub, desc = baseline_sample(job)
    work = oracle.contractions(sub, sub.mask)
    runs, t0 = 0, time.perf_counter()
    while True:
        oracle.compute(sub, mask=sub.mask, with_abs=False)
        runs += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or runs >= max_runs:
            break
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": work * runs / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%s, %d run(s), %.1f s, numpy FP64 (BLAS threads = all cores)" % (desc, runs, el)}


def accuracy_blocks(job):
    """Blocks of the workload the oracle computes one by one for the error report: S, T, V of
    a heavy-heavy and a light-light pair (one-, two- and three-centre V contributions), (P|Q)
    of atoms 0-1, (P|ij) of the last atom's aux on the pair 0-1 grid refined around it."""
    n = job.n_atoms
    pairs = [(0, 1)] + ([(n - 2, n - 1)] if n > 3 else [])
    aux_pairs = [(0, 1)]
    triples = [(n - 1, 0, 1)] if n >= 3 else [(1, 0, 1)]
    return pairs, aux_pairs, triples


def accuracy(job, got):
    """Largest absolute error per class of `got` (host arrays) against the oracle on the
    sampled blocks, and the oracle's seconds."""
    import numpy as np
    import oracle
    pairs, aux_pairs, triples = accuracy_blocks(job)
    t0 = time.perf_counter()
    R = oracle.compute(job, mask=job.mask, with_abs=False, j3_triples=triples, pairs=pairs, aux_pairs=aux_pairs)
    el = time.perf_counter() - t0

    def sl(shells, X):
        off = sum(2 * s[2] + 1 for s in shells if s[0] < X)
        return slice(off, off + sum(2 * s[2] + 1 for s in shells if s[0] == X))

    err = {}
    for k in ("S", "T", "V"):
        if k in got:
            err[k] = max(float(np.abs(got[k][sl(job.basis, A), sl(job.basis, B)] -
                                       R[k][sl(job.basis, A), sl(job.basis, B)]).max()) for A, B in pairs)
    if "J2" in got:
        err["J2"] = max(float(np.abs(got["J2"][sl(job.aux, C), sl(job.aux, D)] -
                                      R["J2"][sl(job.aux, C), sl(job.aux, D)]).max()) for C, D in aux_pairs)
    if "J3" in got:
        err["J3"] = max(float(np.abs(got["J3"][sl(job.aux, C), sl(job.basis, A), sl(job.basis, B)] -
                                      R["J3"][sl(job.aux, C), sl(job.basis, A), sl(job.basis, B)]).max())
                        for C, A, B in triples)
    desc = "oracle blocks: S/T/V %s, J2 %s, J3 (aux atom, i atom, j atom) %s" % (pairs, aux_pairs, triples)
    return err, desc, el


def line_config(job, args, world=1):
    """The `config` of both arms' lines (the same dict: workload, sizes, precision, L2 note)."""
    return {"workload": args.workload, "seed": args.seed, "precision": args.precision, "n_bf": job.n_bf,
            "n_aux": job.n_aux, "classes": "S,T,V,J2,J3" if job.mask == 31 else job.mask,
            "l2": "working set above the 129 MB L2 (no flush needed)",
            "parallelism": "replicas" if world > 1 else "single"}


def default_steps(args):
    if args.steps is not None:
        return args.steps
    return {"triatomic_oh2": 400, "h2_fp64": 400}.get(args.workload, 10)


def reference_arm(args):
    """The CPU oracle, as it stands, on the host cores: each step is the oracle_sample of the
    workload (atoms 0-1, one pair grid, every class)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth
    job = synth.WORKLOADS[args.workload](args.seed)
    sub, desc = oracle_sample(job)
    work = oracle.contractions(sub, sub.mask)
    steps = default_steps(args)
    for _ in range(args.warmup):
        oracle.compute(sub, mask=sub.mask, with_abs=False)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.compute(sub, mask=sub.mask, with_abs=False)
    el = time.perf_counter() - t0
    value = work * steps / el
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": line_config(job, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------ clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        """Starts sampling every 200 ms and returns once the first sample is written (so the
        timed region that follows is covered from its start)."""
        self.skip = 0
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
            self.skip = sum(1 for _ in open(self.path))  # samples taken before the region
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        lines = open(self.path).readlines()
        # the samples inside the timed region (the last one before it if the region was shorter
        # than the sampling period)
        for line in lines[max(0, min(self.skip, len(lines) - 1)):]:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------ RI timing

def time_ri(J2, J3, stream, reps=20):
    """Device time of the RI 4-index assembly (eq 14) on the job's own (P|Q) and (P|ij): Cholesky
    factor, forward solve of all pairs, then (ij|kl) for the first min(pairs, 4096) pairs
    against each other (FP64 CUDA cores), replayed from a captured CUDA graph."""
    import torch
    import paper_2510_15204_gb300 as P
    n = J2.shape[0]
    B = torch.empty((n, J3.numel() // max(n, 1)), dtype=torch.float64, device=J3.device)
    m = B.shape[1]
    mb = min(m, 4096)
    eri = torch.empty((mb, mb), dtype=torch.float64, device=J3.device)
    L = torch.empty_like(J2)

    info_box = []

    def once():
        _, info = P.ri_factor(J2, L=L, stream=stream)
        info_box.append(info)
        B.copy_(J3.reshape(n, m))
        P.ri_solve(L, B, stream=stream)
        P.ri_eri(B, 0, mb, 0, mb, out=eri, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(3):
            once()
        torch.cuda.synchronize()
        # replayed from a CUDA graph: the ~20 small launches of a small job would otherwise
        # wait on the host between them
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            once()
        graph.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = n ** 3 / 3.0 + float(n) * n * m + 2.0 * n * mb * mb

    # the (ij|kl) block alone: FP64 CUDA cores against the tensor-core (8-bit slice) product
    need = ctypes.c_size_t()
    P.lib().psq_ri_eri_mixed_workspace(n, mb, mb, ctypes.byref(need))
    wsm = torch.empty(max(256, need.value), dtype=torch.uint8, device=J3.device)
    emx = torch.empty_like(eri)

    def timed(fn, k=5):
        with torch.cuda.stream(stream):
            fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(k):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    t64 = timed(lambda: P.ri_eri(B, 0, mb, 0, mb, out=eri, stream=stream))
    tmx = timed(lambda: P.ri_eri_mixed(B, 0, mb, 0, mb, out=emx, ws=wsm, stream=stream))
    dev = float((emx - eri).abs().max() / eri.abs().max())
    info = int(info_box[0].item())  # 0: this (P|Q) factored (it is positive definite at FP64)
    if not math.isfinite(dev):
        dev = None  # a metric that did not factor leaves B undefined (and NaN is not JSON)
    eflops = 2.0 * n * mb * mb
    return {"ms": ms, "n_aux": n, "pairs": m, "eri_pairs": mb, "factor_info": info,
            "fp64_flop": flops, "tflops": flops / (ms / 1e3) / 1e12,
            "peak": FP64_PEAK_TFLOPS, "peak_source": "nominal GB300 FP64",
            "eri_block": {"fp64_ms": t64, "fp64_tflops": eflops / (t64 / 1e3) / 1e12, "tensor_ms": tmx,
                          "tensor_useful_tflops": eflops / (tmx / 1e3) / 1e12, "tensor_max_dev_rel": dev}}


# ------------------------------------------------------------------------------ traffic record

def recorded_traffic(kernel, workload, precision):
    """DRAM bytes of `kernel` per bench step from profiles/traffic.txt, if recorded for the current
    sources of the kernel and its planner (null once either changed since the counters were
    taken)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split("#")[0].split()
        if len(f) != 6 or f[0] != kernel or f[1] != workload or f[2] != precision:
            continue
        # the kernel's source files (joined by "+": the kernel and the planner that shapes
        # its launches), hashed together
        srcs = [os.path.join(ROOT, "paper_2510_15204_gb300", "csrc", n) for n in f[3].split("+")]
        if all(os.path.exists(x) for x in srcs):
            h = hashlib.sha256(b"".join(open(x, "rb").read() for x in srcs)).hexdigest()[:16]
            if h == f[4]:
                return int(f[5])
    return None


# ------------------------------------------------------------------------------ serving

def serve_block(P, ctx, args, rate=20.0, n_jobs=60, n_fp64=3):
    """A short serving run for the bench line: a Poisson stream of random molecules (2..9
    atoms, DZ/TZ/QZ-sized bases, config-2 grids) through the continuous-batching server on the
    mixed path, and the stream's first jobs as per-job plain FP64 launches (FIFO)."""
    import threading
    import numpy as np
    import torch
    import synth
    mask = P.ALL
    stream = synth.serving_stream(seed=args.seed, rate=rate, n_jobs=n_jobs)
    jobs = [P.Job.from_synth(ctx, j, P.MIXED) for _, j in stream]
    outs = [{k: torch.empty(sh, dtype=torch.float64).pin_memory() for k, sh in J.out_shapes(mask).items()}
            for J in jobs]
    for J in jobs:
        J.workspace_bytes(mask)  # plan up front: planning is host work, not serving latency
    work = sum(J.stats(mask)["contractions"] for J in jobs)
    server = P.Server(ctx, arena_bytes=int(torch.cuda.mem_get_info()[0] * 0.5), max_inflight=6)
    tickets = [None] * len(jobs)
    t0 = time.perf_counter()

    def feeder():
        for i, (t_arr, _) in enumerate(stream):
            d = t0 + t_arr - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets[i] = server.submit(jobs[i], mask, outs[i])

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    lat = [server.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    server.close()
    res = {"rate_per_s": rate, "jobs": len(jobs), "p50_s": float(np.percentile(lat, 50)),
           "p99_s": float(np.percentile(lat, 99)), "jobs_per_s": len(jobs) / wall,
           "contractions_per_s": work / wall, "precision": "mixed (1e-9 absolute)"}
    lat64, busy, t_gpu = [], 0.0, 0.0
    stream64 = stream[:n_fp64]
    work64 = 0.0
    for (t_arr, j) in stream64:
        J = P.Job.from_synth(ctx, j, P.FP64)
        work64 += J.stats(mask)["contractions"]
        ws, out = J.alloc(mask)
        host = {k: torch.empty(v.shape, dtype=torch.float64).pin_memory() for k, v in out.items()}
        t1 = time.perf_counter()
        J.compute_host(mask, ws, out, host)
        dt = time.perf_counter() - t1
        t_gpu += dt
        start = max(t_arr, busy)
        busy = start + dt
        lat64.append(busy - t_arr)
        del ws, out
        torch.cuda.empty_cache()
    res["fp64_per_job"] = {"jobs": len(stream64), "p50_s": float(np.percentile(lat64, 50)),
                           "p99_s": float(np.percentile(lat64, 99)), "contractions_per_s": work64 / t_gpu,
                           "note": "the stream's first jobs, one launch sequence per job, FIFO"}
    return res


def serve_main(args):
    """Poisson stream of random molecules (2..9 atoms, Z in {1,6,7,8}, DZ/TZ/QZ-sized bases,
    config-2 grids) through the continuous-batching server (mixed precision, within 1e-9 of
    the FP64 oracle), swept over arrival rates, against the same stream's first jobs run one by
    one on the plain FP64 path.  Latency is from a job's arrival to its results in host memory
    (host queueing included); p99 over the rate's jobs (--jobs, 300 by default)."""
    import threading
    import numpy as np
    import torch
    import synth
    from paper_2510_15204_gb300 import build as B
    B.build()
    import paper_2510_15204_gb300 as P
    torch.cuda.set_device(0)
    ctx = P.Context(0)
    mask = P.ALL
    res = {"metric": "serve p50/p99 latency and throughput", "unit": "s", "higher_is_better": False,
           "data": "synthetic", "n_gpus": 1, "rates": []}
    arena_bytes = int(torch.cuda.mem_get_info()[0] * 0.6)
    server = P.Server(ctx, arena_bytes=arena_bytes, max_inflight=6)
    for rate in [float(x) for x in args.rates.split(",")]:
        stream = synth.serving_stream(seed=args.seed, rate=rate, n_jobs=args.jobs)
        jobs = [P.Job.from_synth(ctx, j, P.MIXED) for _, j in stream]
        for J in jobs:
            J.workspace_bytes(mask)  # plan up front: planning is host work, not serving latency
        work = sum(J.stats(mask)["contractions"] for J in jobs)
        n = len(jobs)
        tickets, outs, sub_t = [None] * n, [None] * n, [0.0] * n
        lat = [0.0] * n
        state = {"done": 0}
        cv = threading.Condition()
        window = args.serve_window
        t0 = time.perf_counter()

        def feeder():
            # jobs arrive at their stream times; at most `window` are submitted and unfinished
            # (the rest wait on the host, inside their measured latency); each job's pinned
            # result buffers exist from its submission to its completion
            try:
                for i, (t_arr, _) in enumerate(stream):
                    with cv:
                        while i - state["done"] >= window and "error" not in state:
                            cv.wait()
                    if "error" in state:
                        return
                    out = {k: torch.empty(sh, dtype=torch.float64).pin_memory()
                           for k, sh in jobs[i].out_shapes(mask).items()}
                    d = t0 + t_arr - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    outs[i] = out
                    sub_t[i] = time.perf_counter()
                    t = server.submit(jobs[i], mask, out)
                    with cv:
                        tickets[i] = t
                        cv.notify_all()
            except Exception as e:  # let the collector stop too
                with cv:
                    state["error"] = repr(e)
                    cv.notify_all()

        def collector():
            try:
                for i in range(n):
                    with cv:
                        while tickets[i] is None and "error" not in state:
                            cv.wait()
                    if "error" in state:
                        return
                    served = server.wait(tickets[i])  # submission -> results in host memory
                    lat[i] = (sub_t[i] - (t0 + stream[i][0])) + served
                    outs[i] = None
                    with cv:
                        state["done"] += 1
                        cv.notify_all()
            except Exception as e:
                with cv:
                    state["error"] = repr(e)
                    cv.notify_all()

        threads = [threading.Thread(target=feeder), threading.Thread(target=collector)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        if "error" in state:
            raise RuntimeError("serving run failed: " + state["error"])
        wall = max(stream[i][0] + lat[i] for i in range(n))  # arrival of the first job at 0
        res["rates"].append({"rate_per_s": rate, "jobs": len(jobs), "p50_s": float(np.percentile(lat, 50)),
                             "p99_s": float(np.percentile(lat, 99)), "throughput_jobs_per_s": len(jobs) / wall,
                             "contractions_per_s": work / wall, "precision": "mixed (1e-9 absolute)"})
        sys.stderr.write("rate %g done: p50 %.3f p99 %.3f\n" % (rate, res["rates"][-1]["p50_s"], res["rates"][-1]["p99_s"]))
    server.close()
    # per-job plain FP64 launches, one after another, same arrival times (first jobs of the stream)
    stream = synth.serving_stream(seed=args.seed, rate=float(args.rates.split(",")[0]), n_jobs=args.baseline_jobs)
    jobs = [P.Job.from_synth(ctx, j, P.FP64) for _, j in stream]
    lat, busy_until = [], 0.0
    work = sum(J.stats(mask)["contractions"] for J in jobs)
    t_gpu = 0.0
    for (t_arr, _), J in zip(stream, jobs):
        ws, out = J.alloc(mask)
        host = {k: torch.empty(v.shape, dtype=torch.float64).pin_memory() for k, v in out.items()}
        t1 = time.perf_counter()
        J.compute_host(mask, ws, out, host)
        dt = time.perf_counter() - t1
        t_gpu += dt
        start = max(t_arr, busy_until)  # a single FIFO server of per-job launches
        busy_until = start + dt
        lat.append(busy_until - t_arr)
        del ws, out
        torch.cuda.empty_cache()
    res["fp64_per_job"] = {"jobs": len(jobs), "p50_s": float(np.percentile(lat, 50)),
                           "p99_s": float(np.percentile(lat, 99)), "contractions_per_s": work / t_gpu,
                           "note": "same stream's first jobs, one launch sequence per job, FIFO"}
    print(json.dumps(res))
    return 0


def scan_main(args):
    """The Fig. 6 displacement scans as a throughput workload: every point of every path is
    its own diatomic (P|Q) job, all submitted at once to the continuous-batching server (mixed
    precision); per-job plain FP64 launches on the first jobs beside it, and the largest
    deviation of the served (P|Q) path values from those FP64 values."""
    import numpy as np
    import torch
    import synth
    from paper_2510_15204_gb300 import build as B
    B.build()
    import paper_2510_15204_gb300 as P
    torch.cuda.set_device(0)
    ctx = P.Context(0)
    mask = P.J2
    scan = synth.displacement_scan()
    jobs = [P.Job.from_synth(ctx, j, P.MIXED) for _, j in scan]
    outs = [{k: torch.empty(sh, dtype=torch.float64).pin_memory() for k, sh in J.out_shapes(mask).items()}
            for J in jobs]
    for J in jobs:
        J.workspace_bytes(mask)  # plan up front (host work, not serving latency)
    server = P.Server(ctx, arena_bytes=int(torch.cuda.mem_get_info()[0] * 0.5), max_inflight=8)
    t0 = time.perf_counter()
    tickets = [server.submit(J, mask, o) for J, o in zip(jobs, outs)]
    lat = [server.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    server.close()
    n_fp64 = min(args.baseline_jobs * 50, len(jobs))
    dev, t_gpu = 0.0, 0.0
    for (meta, j), o in zip(scan[:n_fp64], outs[:n_fp64]):
        J = P.Job.from_synth(ctx, j, P.FP64)
        ws, out = J.alloc(mask)
        host = {k: torch.empty(v.shape, dtype=torch.float64).pin_memory() for k, v in out.items()}
        t1 = time.perf_counter()
        J.compute_host(mask, ws, out, host)
        t_gpu += time.perf_counter() - t1
        r, c = meta[4], meta[5]
        dev = max(dev, abs(float(o["J2"][r, c]) - float(host["J2"][r, c])))
    res = {"metric": "Fig. 6 displacement scans through the serving loop", "unit": "jobs/s", "higher_is_better": True,
           "data": "synthetic", "n_gpus": 1,
           "config": {"workload": "displacement_scan", "paths": len(synth.SCAN_PAIRS) * 16, "points_per_path": 51,
                      "pairs_l": synth.SCAN_PAIRS, "grid": list(scan[0][1].specs[0]), "precision": "mixed"},
           "jobs": len(jobs), "value": len(jobs) / wall, "wall_s": wall,
           "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "fp64_per_job": {"jobs": n_fp64, "jobs_per_s": n_fp64 / t_gpu},
           "max_abs_dev_vs_fp64": dev}
    print(json.dumps(res))
    return 0


# ------------------------------------------------------------------------------ GPU arm

def ri_main(args):
    """The RI 4-index assembly (eq 14) alone, on seeded synthetic matrices of a job's shape: a
    symmetric positive definite (P|Q) = X X^T / n + I and a normal (P|ij); factor, solve of all
    pair columns and the first min(m, 4096)^2 block of (ij|kl), FP64 and on the tensor cores."""
    import torch
    from paper_2510_15204_gb300 import build as B
    B.build()
    n, m = (int(x) for x in args.ri_sizes.split(","))
    torch.cuda.set_device(0)
    g = torch.Generator(device="cuda").manual_seed(args.seed)
    X = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    J2 = X @ X.T / n + torch.eye(n, dtype=torch.float64, device="cuda")
    J3 = torch.randn((n, m), dtype=torch.float64, device="cuda", generator=g)
    stream = torch.cuda.Stream()
    res = time_ri(J2, J3, stream)
    print(json.dumps({"metric": "RI 4-index assembly (eq 14), synthetic matrices", "unit": "ms", "n_aux": n,
                      "pairs": m, "ri_4index": res, "data": "synthetic", "seed": args.seed}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.ri_sizes:
        return ri_main(args)
    if args.serve:
        return serve_main(args)
    if args.scan:
        return scan_main(args)
    rank, world, local = dist_env()
    import torch
    import synth
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2510_15204_gb300 import build as B
    B.build()
    import paper_2510_15204_gb300 as P

    job = synth.WORKLOADS[args.workload](args.seed)
    mask = job.mask
    args.steps = default_steps(args)
    ctx = P.Context(local)
    prec = P.MIXED if args.precision == "mixed" else P.FP64
    J = P.Job.from_synth(ctx, job, prec)
    ws, out = J.alloc(mask, headroom=0.25)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        # the work split is tuned on this job during warm-up (candidates that fit the workspace)
        tuned = None
        if not args.no_autotune:
            split, tms = J.autotune(mask, ws, out, stream)
            tuned = {"work_split": split, "ms": tms}
        for _ in range(max(args.warmup, 3)):
            J.compute(mask, ws, out, stream)
    torch.cuda.synchronize()
    st = J.stats(mask)
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    J.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        J.compute(mask, ws, out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    J.profile(False)
    prof = J.profile_read()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    (t_max,), (value,) = aggregate([ms / 1e3], [st["contractions"] * args.steps], world)
    ms = t_max * 1e3
    if world > 1:
        dist.barrier()

    # the same steps replayed from the job's captured CUDA graph
    graph = None
    if not args.no_graph:
        with torch.cuda.stream(stream):
            J.compute_graph(mask, ws, out, stream)
            torch.cuda.synchronize()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(args.steps):
                J.compute_graph(mask, ws, out, stream)
            g1.record(stream)
            torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / args.steps
        graph = {"ms_per_step": gms, "value": st["contractions"] / (gms / 1e3)}

    # the plain FP64 path on the same job ("vs plain FP64"), a few steps
    plain = None
    host_mixed = {k: v.cpu().numpy() for k, v in out.items()}
    if prec == P.MIXED and args.fp64_steps > 0:
        J64 = P.Job.from_synth(ctx, job, P.FP64)
        ws64, out64 = J64.alloc(mask)
        with torch.cuda.stream(stream):
            J64.compute(mask, ws64, out64, stream)
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(args.fp64_steps):
                J64.compute(mask, ws64, out64, stream)
            f1.record(stream)
            torch.cuda.synchronize()
        fms = f0.elapsed_time(f1) / args.fp64_steps
        # every element of the mixed result against the plain FP64 GPU path (itself within 1e-12
        # of the oracle's absolute-term sums in the tests)
        dev = {k: float((out64[k].cpu() - torch.from_numpy(host_mixed[k])).abs().max()) for k in out}
        plain = {"value": st["contractions"] / (fms / 1e3), "ms_per_step": fms, "steps": args.fp64_steps,
                 "speedup_of_mixed": fms / (ms / args.steps), "workspace_gb": J64.workspace_bytes(mask) / 1e9,
                 "max_abs_dev_of_mixed_every_element": dev}
        del ws64, out64, J64
        torch.cuda.empty_cache()
    acc = None
    if prec == P.MIXED and not args.no_accuracy and rank == 0:
        err, desc, osec = accuracy(job, host_mixed)
        acc = {"max_abs_err_vs_oracle": err, "target": 1e-9, "met": all(v <= 1e-9 for v in err.values()),
               "blocks": desc, "oracle_s": osec}

    # end to end through the C ABI with host buffers (tables up, matrices down, every step)
    host = {k: torch.empty(v.shape, dtype=torch.float64).pin_memory() for k, v in out.items()}
    with torch.cuda.stream(stream):
        J.compute_host(mask, ws, out, host, stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            J.compute_host(mask, ws, out, host, stream)
        e2e_s = time.perf_counter() - t0
    h2d, d2h = J.io_bytes(mask)
    _, (e2e_val,) = aggregate([e2e_s], [st["contractions"] * args.e2e_steps], world)

    # RI 4-index assembly (eq 14) on this step's (P|Q) and (P|ij): factor, solve, all (ij|kl)
    ri = None
    if "J2" in out and "J3" in out and not args.no_ri:
        ri = time_ri(out["J2"], out["J3"], stream)

    # this device's FP64 / FP32 FMA and SFU rates, measured by the library's probe (after the
    # timed region; context for the FP64- and FP32-bound kernels)
    try:
        mpeaks = P.measure_peaks(stream)
        mpeaks["method"] = "psq_measure_peaks: dependent FMA / ex2.approx chains, fastest of 3 launches"
    except P.PsqError as exc:
        mpeaks = {"error": str(exc)}

    # roofline of the dominant kernel, timed live inside the timed region
    kind = max(prof, key=lambda k: prof[k][0])
    kms, kcount = prof[kind]
    # (per launch: the summed time of the kind over the step's launches, i.e. per step)
    per_launch_s = kms / args.steps / 1e3
    if kind == "contract":
        flops = 2.0 * st["contractions"]
        if prec == P.FP64:
            # the nominal rate stays the ceiling: the dependent-chain probe reads below what
            # eri_kernel sustains on the same pipe
            roof = {"bound": "alu", "achieved": flops / per_launch_s / 1e12, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "peak_source": "nominal GB300 FP64",
                    "peak_probe": mpeaks.get("fp64_tflops")}
        else:
            # achieved counts the method's work (2 FLOPs per useful contraction); the tensor pipe
            # issues 15 slice products per useful product on padded 128 x 48 tiles
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
            issued = st["issued_flops"] / per_launch_s / 1e12
            roof = {"bound": "tensor", "achieved": flops / per_launch_s / 1e12,
                    "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "peak_source": "measured bf16 burst",
                    "counts": "useful FLOPs (2 per contraction)",
                    "issued_tflops": issued, "issued_frac": issued / peaks["bf16_tflops"],
                    "issued_counts": "bf16 MMA FLOPs issued: 15 slice products of 128 x 48 x 32 per item and chunk"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s"}
    roof["kernel"] = kind
    roof["launches_per_step"] = kcount / args.steps
    roof["frac"] = roof["achieved"] / roof["peak"] if roof.get("achieved") else None
    # DRAM bytes per launch (the step's recorded bytes over its launches, as `achieved` is the
    # step's work over its launches' time), and per step
    step_bytes = recorded_traffic(kind, args.workload, args.precision)
    roof["traffic"] = step_bytes / roof["launches_per_step"] if step_bytes and roof["launches_per_step"] else None
    roof["traffic_per_step"] = step_bytes
    roof["share"] = kms / sum(v[0] for v in prof.values())

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == P.FP64 else "double-float (2 x f32) values, bf16 8-bit slices, f32/f64 sums",
        "data": "synthetic",
        "config": line_config(job, args, world),
        "job": {"grids": st["grids"], "points": st["points"], "contractions_per_step": st["contractions"],
                "workspace_gb": J.workspace_bytes(mask) / 1e9, "launches_per_step": st["launches"]},
        "accuracy": acc,
        "roofline": roof,
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "graph": graph,
        "autotune": tuned,
        "plain_fp64": plain,
        "ri_4index": ri,
        "gpu_launches": st["launches"] * args.steps,
        "clocks": clk,
        "measured_peaks": mpeaks,
    }
    if rank == 0 and world == 1 and not args.no_serve_block and prec == P.MIXED:
        line["serve"] = serve_block(P, ctx, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = time_oracle(job)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
