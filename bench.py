#!/usr/bin/env python3
"""Benchmark of the GB300 PC-LSQR (Gaia AVU-GSR hot path).

One step = one whole PC-LSQR solve through the C ABI (preconditioner, the
LSQR iterations with aprod 1 / aprod 2 and the vector updates, the final
x = p o z and standard errors) on a synthetic system of the paper's
structure.  The metric is LSQR iterations per second over the whole job.

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
replica (different seed, same shape): the path needs no exchange between
replicas, so there is no collective on the data path ("scaling": "weak").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload medium]
  python bench.py --impl reference ...   # the CPU oracle, timed on host cores
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2212_11675_gb300 import gen  # noqa: E402

ITMAX = {"tiny": 200, "medium": 500}
METRIC = "PC-LSQR iter/s"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# sources of the row kernels; a capture's DRAM traffic applies only while
# their hash is the one recorded beside it
KERNEL_SOURCES = ("gsr_kernels.cu", "gsr_internal.cuh", "gsr_split.cuh", "gsr_reduce.cuh")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2212_11675_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel, workload):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    summaries under profiles/: a line
      traffic: <kernel> workload=<w> dram_bytes_per_launch=<B> source_sha256=<h>
    counts only while <h> is the hash of the current kernel sources (None
    otherwise, or when no capture of this kernel and workload is recorded)."""
    import glob
    import re
    want = kernel_source_hash()
    pat = re.compile(r"^traffic:\s+(\S+)\s+workload=(\S+)\s+dram_bytes_per_launch=(\S+)\s+"
                     r"source_sha256=([0-9a-f]+)")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for ln in f:
                m_ = pat.match(ln.strip().strip("`"))
                if m_ and m_.group(1) == kernel and m_.group(2) == workload and m_.group(4) == want:
                    return float(m_.group(3)), os.path.relpath(path, ROOT)
    return None, None


def fp64_fma_rate():
    """FP64 FMAs per second of this GPU, measured now by the library's probe."""
    import ctypes
    from paper_2212_11675_gb300 import _lib
    r = ctypes.c_double(0.0)
    _lib.check(_lib.lib().gsr_fp64_fma_rate(ctypes.byref(r)), "gsr_fp64_fma_rate")
    return r.value


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([c.strip() for c in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def whole_job(iters, t, dist, dev, torch):
    """Replicas: the iterations of all ranks and the slowest rank's time (the
    whole job's throughput is their ratio); one rank without dist."""
    if not dist:
        return float(iters), float(t)
    it_all = torch.tensor([float(iters)], dtype=torch.float64, device=dev)
    t_all = torch.tensor([float(t)], dtype=torch.float64, device=dev)
    dist.all_reduce(it_all, op=dist.ReduceOp.SUM)
    dist.all_reduce(t_all, op=dist.ReduceOp.MAX)
    return float(it_all), float(t_all)


def make_system(workload, rank):
    shape = gen.SHAPES[workload]
    seed = gen.SEEDS[workload] + 7919 * rank
    return gen.generate(shape, seed), seed


def run_reference(args):
    """The CPU oracle, as it stands, on a bounded sample of the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    sys_, seed = make_system(args.workload, 0)
    xt = gen.x_true(sys_, seed)
    b = oracle.aprod1(sys_, xt) + gen.noise(sys_, seed + 1)
    iters = args.ref_iters
    for _ in range(args.warmup):
        oracle.pc_lsqr(sys_, b, 1, 0.0, 0.0)
    t0 = time.perf_counter()
    total = 0
    for _ in range(args.steps):
        r = oracle.pc_lsqr(sys_, b, iters, 0.0, 0.0)
        total += r["itn"]
    dt = time.perf_counter() - t0
    val = total / dt
    sample = ("%d steps x (preconditioner + %d LSQR iterations) of the %s system (m=%d, n=%d)"
              % (args.steps, iters, args.workload, sys_.m, sys_.n))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "iter/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "m": sys_.m, "n": sys_.n},
            "cpu_baseline": {"value": val, "unit": "iter/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_kernel(fn, stream, reps, torch):
    """Average duration (s) of fn() launched reps times on `stream`."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps * 1e-3


# stopping tolerances tried from loose to tight: the loosest one that meets
# the accuracy target is the fastest setting of that form
TOL_LADDER = (1e-6, 3e-7, 1e-7, 3e-8, 1e-8, 3e-9, 1e-9, 3e-10, 1e-10, 3e-11, 1e-11, 1e-12)


def _timer(torch, stream, reps):
    def timed(fn):
        best, out = None, None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best, out
    return timed


def _rel(torch, x, xr):
    torch.cuda.synchronize()  # x may come from a solve on another stream
    return float(torch.linalg.norm(x - xr) / torch.linalg.norm(xr))


def time_to_solution(s, b, torch, stream, target=1e-9, reps=3):
    """Time for the FP64 PC-LSQR and for the mixed-precision solve to reach a
    solution within `target` (relative) of the FP64 least-squares solution,
    on the same GPU and the same mixed-precision solver `s` (which holds both
    the FP64 and the binary32 matrix).  Each form runs its tolerance ladder
    from loose to tight; the fastest setting that meets the target is
    reported (FP64: the loosest atol = btol that meets it; mixed: over the
    outer atol and the inner CG tolerance)."""
    timed = _timer(torch, stream, reps)
    res = {"target_rel_err": target, "ladder": "atol from 1e-6 down"}
    xr, _, rr = s.lsqr_solve(b, 20000, 1e-15, 1e-15, stream=stream, want_se=False)
    res["reference"] = {"itn": rr["itn"], "istop": rr["istop"], "atol": 1e-15}
    best = None
    for tol in TOL_LADDER:
        ms, out = timed(lambda: s.lsqr_solve(b, 20000, tol, tol, stream=stream, want_se=False))
        err = _rel(torch, out[0], xr)
        if err <= target:
            best = {"ms": ms, "itn": out[2]["itn"], "atol": tol, "rel_err": err}
            break
    res["fp64"] = best
    bestm, first_ok = None, None
    for i, tol in enumerate(TOL_LADDER):
        for itol in (1e-2, 1e-3, 1e-4):
            ms, out = timed(lambda: s.mixed_solve(b, max_outer=30, max_inner=500,
                                                  inner_tol=itol, atol=tol, stream=stream))
            err = _rel(torch, out[0], xr)
            if err <= target and (bestm is None or ms < bestm["ms"]):
                bestm = {"ms": ms, "outer": out[1]["outer"], "inner": out[1]["inner"],
                         "atol": tol, "inner_tol": itol, "rel_err": err}
        if bestm is not None and first_ok is None:
            first_ok = i
        if first_ok is not None and i >= first_ok + 1:  # one step past the first success
            break
    res["mixed"] = bestm
    if best and bestm:
        res["speedup"] = best["ms"] / bestm["ms"]
    return res


def batched_vs_sequential(s, xt, noise, torch, stream, ks=(8, 32), target=1e-9, reps=1,
                          ref_tol=1e-13):
    """Time for the batched k-RHS solve to bring every column within `target`
    of its FP64 least-squares solution, against k sequential FP64 PC-LSQR
    solves at the loosest tolerance that meets the same target on every
    column.  Right-hand side j is A xt + noise(j) (independent noise streams).
    The FP64 references (atol = btol = ref_tol) and the sequential solves run once
    for the largest k; the first k of them serve each smaller k (the
    sequential time of k columns is read from events inside that run)."""
    from paper_2212_11675_gb300 import autotune
    timed = _timer(torch, stream, reps)
    out = {"target_rel_err": target, "ladder": "atol from 1e-6 down"}
    K = max(ks)
    ax = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()  # xt and ax come from the current stream, the solves use `stream`
    s.aprod1(xt, ax, stream=stream)
    torch.cuda.synchronize()
    B = torch.empty((K, s.m), dtype=torch.float64, device="cuda")
    for j in range(K):
        torch.add(ax, noise(j), out=B[j])
    torch.cuda.synchronize()
    del ax
    refs = [s.lsqr_solve(B[j], 20000, ref_tol, ref_tol, stream=stream, want_se=False)[0]
            for j in range(K)]
    out["reference_atol"] = ref_tol
    # sequential FP64: the loosest ladder tolerance meeting the target on column
    # 0, then on every column (tightened while a column misses it)
    tol_i = 0
    for tol_i, tol in enumerate(TOL_LADDER):
        x0 = s.lsqr_solve(B[0], 20000, tol, tol, stream=stream, want_se=False)[0]
        if _rel(torch, x0, refs[0]) <= target:
            break
    seq = None
    while tol_i < len(TOL_LADDER):
        tol = TOL_LADDER[tol_i]
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        ev[0].record(stream)
        xs = []
        for j in range(K):
            xs.append(s.lsqr_solve(B[j], 20000, tol, tol, stream=stream, want_se=False)[0])
            ev[j + 1].record(stream)
        torch.cuda.synchronize()
        errs = [_rel(torch, xs[j], refs[j]) for j in range(K)]
        if max(errs) <= target:
            seq = {"atol": tol, "ms": {k: ev[0].elapsed_time(ev[k]) for k in ks},
                   "max_rel_err": {k: max(errs[:k]) for k in ks}}
            break
        tol_i += 1
    del xs
    for k in ks:
        torch.cuda.empty_cache()
        kt, lanes, tune = autotune.tune(s, k)
        bat = None
        for tol in TOL_LADDER:
            s.batched_solve(B[:k], max_outer=30, max_inner=500, inner_tol=1e-3, atol=tol,
                            stream=stream)  # graph build and warm-up
            ms, (X, res) = timed(lambda: s.batched_solve(B[:k], max_outer=30, max_inner=500,
                                                         inner_tol=1e-3, atol=tol, stream=stream))
            err = max(_rel(torch, X[j], refs[j]) for j in range(k))
            if err <= target:
                bat = {"ms": ms, "atol": tol, "inner_tol": 1e-3, "max_rel_err": err,
                       "outer": max(r["outer"] for r in res), "inner": max(r["inner"] for r in res)}
                break
        sq = ({"ms": seq["ms"][k], "atol": seq["atol"], "max_rel_err": seq["max_rel_err"][k]}
              if seq else None)
        out["k%d" % k] = {"sequential_fp64": sq, "batched": bat,
                          "tiling": {"kt": kt, "lanes": lanes},
                          "speedup": (sq["ms"] / bat["ms"]) if (sq and bat) else None}
    return out


def large_comparison(name, torch, stream, ks=(8, 32)):
    """Time to solution on a large workload generated on the device: the
    mixed-precision solve against FP64 PC-LSQR (1,000,000 stars), or the
    batched k-RHS solve against k sequential FP64 solves (2,000,000 stars)."""
    from paper_2212_11675_gb300 import _lib
    from paper_2212_11675_gb300.solver import Solver
    dev = torch.device("cuda", torch.cuda.current_device())
    seed = gen.SEEDS[name]
    t0 = time.perf_counter()
    sys_ = gen.make_t(name, dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    m, n = sys_.m, sys_.n
    cfg = {"workload": name, "stars": sys_.n_stars, "m": m, "n": n, "n_dfa": sys_.n_dfa,
           "n_instr": sys_.n_instr, "nnz": 24 * m, "generated_on": "device"}
    t0 = time.perf_counter()
    s = Solver(sys_, conlim=0.0, precision=_lib.GSR_PREC_MIXED, validate=False)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    sys_.values = None
    sys_.instr = sys_.attoff = None
    torch.cuda.empty_cache()
    xt = gen.x_true_t(sys_, seed, dev)
    line = {"config": cfg, "generate_s": t_gen, "create_s": t_create,
            "device_bytes": s.device_bytes,
            "dtype": "f32 storage, f64 accumulation and refinement"}
    try:
        with Clocks(torch.cuda.current_device()) as clk:
            if name == "large":
                b = gen.noise_t(sys_, seed + 1, dev)
                torch.cuda.synchronize()  # b and xt come from the current stream
                s.aprod1(xt, b, stream=stream)
                torch.cuda.synchronize()
                line["mixed_vs_fp64"] = time_to_solution(s, b, torch, stream, reps=2)
            else:
                line["batched_vs_sequential_fp64"] = batched_vs_sequential(
                    s, xt, lambda j: gen.noise_t(sys_, seed + 1000 * (j + 1), dev), torch,
                    stream, ks=tuple(ks), ref_tol=1e-12)
        line["clocks"] = clk.summary()
    finally:
        s.close()
        del sys_, xt
        torch.cuda.empty_cache()
    return line


def tts_main(args):
    """Only the time-to-solution comparison on one large workload."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    line = large_comparison(args.tts, torch, stream, ks=args.tts_k)
    line["metric"] = "time to 1e-9 relative error vs the FP64 least-squares solution"
    line["unit"] = "ms"
    line["higher_is_better"] = False
    print(json.dumps(line), flush=True)
    return 0


def profile_main(args):
    """A short run of the mixed-precision or batched path on the medium
    workload with host-launched kernels (eager), for ncu: ncu does not profile
    kernel nodes inside graphs with conditional nodes."""
    import torch
    from paper_2212_11675_gb300 import _lib
    from paper_2212_11675_gb300.solver import Solver
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    sys_, seed = make_system(args.workload, 0)
    out = {"profile": args.profile, "workload": args.workload}
    with Solver(sys_, conlim=0.0, precision=_lib.GSR_PREC_MIXED, eager=True) as s:
        xt = torch.tensor(gen.x_true(sys_, seed), device=dev)
        b = torch.tensor(gen.noise(sys_, seed + 1), device=dev)
        s.aprod1(xt, b, stream=stream)
        torch.cuda.synchronize()
        if args.profile == "mixed":
            for _ in range(2):
                _, r = s.mixed_solve(b, max_outer=1, max_inner=10, inner_tol=0.0, atol=0.0,
                                     stream=stream)
            out["result"] = r
        else:
            k = args.profile_k
            g = torch.Generator(device=dev).manual_seed(1)
            X = torch.randn((k, s.n), dtype=torch.float64, device=dev, generator=g)
            Y = torch.randn((k, s.m), dtype=torch.float64, device=dev, generator=g)
            s.set_batch_tiling(args.profile_kt, args.profile_lanes)
            torch.cuda.synchronize()  # X and Y come from the current stream
            for _ in range(2):
                s.batched_products(X, Y, stream=stream)
            B = b.repeat(k, 1)
            torch.cuda.synchronize()
            _, r = s.batched_solve(B, max_outer=1, max_inner=10, inner_tol=0.0, atol=0.0,
                                   stream=stream)
            out["result"] = r[0]
        torch.cuda.synchronize()
    print(json.dumps(out), flush=True)
    return 0


def cpu_baseline_openmp(sys_, seed, seconds):
    """The multi-threaded (OpenMP) CPU PC-LSQR on all host cores, a second
    reported baseline (not the oracle), on a bounded sample as cpu_baseline."""
    import oracle
    xt = gen.x_true(sys_, seed)
    b = oracle.aprod1(sys_, xt) + gen.noise(sys_, seed + 1)
    t0 = time.perf_counter()
    oracle.omp_pc_lsqr(sys_, b, 1, 0.0, 0.0)
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.omp_pc_lsqr(sys_, b, 5, 0.0, 0.0)
    per_it = max((time.perf_counter() - t0 - t1) / 4.0, 1e-6)
    iters = max(1, min(2000, int((seconds - t1) / per_it)))
    # solves (each stops on its own rules) repeated until the time is spent
    t0 = time.perf_counter()
    total, solves = 0, 0
    while True:
        total += oracle.omp_pc_lsqr(sys_, b, iters, 0.0, 0.0)["itn"]
        solves += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return {"value": total / dt, "unit": "iter/s", "cores": oracle.omp_threads(),
            "kind": "openmp",
            "sample": "%d solves (preconditioner + LSQR, %d iterations in all) of the same "
                      "system, OpenMP FP64 C on %d threads (%.1f s)"
                      % (solves, total, oracle.omp_threads(), dt)}


def cpu_baseline(sys_, seed, seconds):
    """The oracle timed on a bounded sample: LSQR iterations of the same system."""
    import oracle
    xt = gen.x_true(sys_, seed)
    b = oracle.aprod1(sys_, xt) + gen.noise(sys_, seed + 1)
    # calibrate: the preconditioner and start cost once, each iteration again
    t0 = time.perf_counter()
    oracle.pc_lsqr(sys_, b, 1, 0.0, 0.0)
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.pc_lsqr(sys_, b, 3, 0.0, 0.0)
    per_it = max((time.perf_counter() - t0 - t1) / 2.0, 1e-6)
    iters = max(1, min(500, int((seconds - t1) / per_it)))
    # solves (each stops on its own rules) repeated until the time is spent
    t0 = time.perf_counter()
    total, solves = 0, 0
    while True:
        total += oracle.pc_lsqr(sys_, b, iters, 0.0, 0.0)["itn"]
        solves += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return {"value": total / dt, "unit": "iter/s", "cores": 1, "kind": "oracle",
            "sample": "%d solves (preconditioner + LSQR, %d iterations in all) of the same "
                      "system, single-threaded FP64 C oracle (%.1f s)" % (solves, total, dt)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="medium", choices=["tiny", "medium"])
    ap.add_argument("--itmax", type=int, default=0)
    ap.add_argument("--ref-iters", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--eager", action="store_true",
                    help="launch the solve's kernels from the host (for ncu, which cannot "
                         "profile kernels inside graphs with conditional nodes)")
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision vs FP64 time-to-solution comparison")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched k-RHS vs sequential FP64 comparison")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 1,000,000-star mixed and 2,000,000-star batched comparisons")
    ap.add_argument("--tts", choices=["large", "xlarge"], default=None,
                    help="only the time-to-solution comparison on a large workload generated "
                         "on the device (large: mixed vs FP64; xlarge: batched vs sequential)")
    ap.add_argument("--tts-k", type=int, nargs="+", default=[8, 32])
    ap.add_argument("--profile", choices=["mixed", "batched"], default=None,
                    help="a short host-launched run of the mixed or batched path (for ncu)")
    ap.add_argument("--profile-k", type=int, default=8)
    ap.add_argument("--profile-kt", type=int, default=8)
    ap.add_argument("--profile-lanes", type=int, default=8)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.tts:
        return tts_main(args)
    if args.profile:
        return profile_main(args)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2212_11675_gb300 import _lib
    from paper_2212_11675_gb300.solver import Solver

    itmax = args.itmax or ITMAX[args.workload]
    sys_, seed = make_system(args.workload, rank)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    solver = Solver(sys_, conlim=0.0, force_itmax=True, eager=args.eager, lanes_per_star=args.lanes)
    # right-hand side b = A x_true + noise, built on the device
    xt = torch.tensor(gen.x_true(sys_, seed), device=dev)
    b = torch.tensor(gen.noise(sys_, seed + 1), device=dev)
    with torch.cuda.stream(stream):
        solver.aprod1(xt, b, stream=stream)
    x = torch.empty(sys_.n, dtype=torch.float64, device=dev)
    se = torch.empty(sys_.n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    def step():
        return solver.lsqr_solve(b, itmax, 0.0, 0.0, x=x, se=se, stream=stream)[2]

    for _ in range(args.warmup):
        step()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    iters = 0
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            iters += step()["itn"]
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    iters_total, t_max = whole_job(iters, t, dist, dev, torch)
    value = iters_total / t_max

    # end to end through the C ABI with host buffers (H2D of b and D2H of x,
    # se inside the timed region), held in pinned (page-locked) host memory as
    # a caller streaming right-hand sides would hold them; the tensors own the
    # memory the NumPy views point into
    b_pin = torch.empty(sys_.m, dtype=torch.float64, pin_memory=True)
    b_pin.copy_(b)
    x_pin = torch.empty(sys_.n, dtype=torch.float64, pin_memory=True)
    se_pin = torch.empty(sys_.n, dtype=torch.float64, pin_memory=True)
    bh, xh, seh = b_pin.numpy(), x_pin.numpy(), se_pin.numpy()
    solver.lsqr_solve(bh, itmax, 0.0, 0.0, x=xh, se=seh, stream=stream)
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(args.steps):
        e2e_iters += solver.lsqr_solve(bh, itmax, 0.0, 0.0, x=xh, se=seh, stream=stream)[2]["itn"]
    e2e_t = time.perf_counter() - t0
    e2e = {"value": ws * e2e_iters / e2e_t, "unit": "iter/s",
           "h2d_bytes_per_step": int(bh.nbytes), "d2h_bytes_per_step": int(xh.nbytes + seh.nbytes)}

    # roofline of the row kernels as they run inside a solve: the launches of
    # 20 LSQR iterations timed with CUDA events on the solve's stream (aprod 1
    # in its LSQR form with ||U||, the single-launch aprod 2 whose partial sums
    # the vector pass combines, the vector pass); each product is also timed
    # alone through its entry point (y += A x, x += A^T y with its combine),
    # for reference
    m, n = sys_.m, sys_.n
    ins = solver.time_iteration(b, iters=20, stream=stream)
    t_a1, t_a2, t_vec = ins["aprod1"] * 1e-3, ins["aprod2"] * 1e-3, ins["vector_pass"] * 1e-3
    yv = torch.zeros(m, dtype=torch.float64, device=dev)
    xv = torch.zeros(n, dtype=torch.float64, device=dev)
    vin = torch.randn(n, dtype=torch.float64, device=dev)
    uin = torch.randn(m, dtype=torch.float64, device=dev)
    reps = 20
    api_a1 = time_kernel(lambda: solver.aprod1(vin, yv, stream=stream), stream, reps, torch)
    api_a2 = time_kernel(lambda: solver.aprod2(uin, xv, stream=stream), stream, reps, torch)
    hbm, src = peaks()
    # algorithmic bytes per launch: 24 values x 8 B + 16 B index record per row,
    # y read+write (aprod 1) or read (aprod 2), 4 B star pointer per star,
    # x gathered / written once per unknown; the vector pass: 11 n-vectors
    # (p, q, v, w, z, var read; w, z, var, v, p o v written)
    bytes_a1 = m * (24 * 8 + 16 + 16) + 4 * sys_.n_stars + 8 * n
    bytes_a2 = m * (24 * 8 + 16 + 8) + 4 * sys_.n_stars + 16 * n
    bytes_vec = 11 * 8 * n
    # FLOPs on the FP64 pipe: one FMA per nonzero, less the products formed on
    # the binary32 pipes from exact splits (7 per row in aprod 1; in aprod 2,
    # 6 per row in the star units, 6 in the instrument units, 4 or 8 in the
    # attitude units)
    split1, split2 = solver.product_forms()
    flops_a1 = 2 * (24 - {0: 0, 1: 7, 2: 12}[split1]) * m
    flops_a2 = 2 * (24 - (6 if split2 & 1 else 0) - (6 if split2 & 2 else 0)
                    - (4 if split2 & 4 else 0) - (8 if split2 & 8 else 0)) * m
    gbs_a1, gbs_a2 = bytes_a1 / t_a1 / 1e9, bytes_a2 / t_a2 / 1e9
    tf_a1, tf_a2 = flops_a1 / t_a1 / 1e12, flops_a2 / t_a2 / 1e12
    dom = "aprod2" if t_a2 >= t_a1 else "aprod1"
    t_dom, gbs_dom, tf_dom, byt = ((t_a2, gbs_a2, tf_a2, bytes_a2) if dom == "aprod2"
                                   else (t_a1, gbs_a1, tf_a1, bytes_a1))
    # DRAM bytes (read + write) per launch of the dominant kernel from the
    # committed ncu capture of the current kernel sources (null when the
    # kernel changed since, or for a workload without a capture)
    kname = {"aprod2": "k_aprod2_fused", "aprod1": "k_aprod1"}[dom]
    traffic, traffic_src = captured_traffic(kname, args.workload)
    fma_rate = fp64_fma_rate()
    fp64_peak = 2.0 * fma_rate / 1e12  # TFLOP/s, measured in this run
    roof = {"bound": "hbm", "achieved": gbs_dom, "peak": hbm, "unit": "GB/s",
            "frac": gbs_dom / hbm, "traffic": traffic, "kernel": kname,
            "peak_source": "%s HBM copy (MEASURED_PEAKS.json)" % src,
            "traffic_source": traffic_src,
            "timing": "in-solve launches (CUDA events, 20 LSQR iterations, host-launched)",
            "algorithmic_bytes_per_launch": byt,
            "fp64_pipe": {"achieved_TFLOP/s": tf_dom, "peak_TFLOP/s": fp64_peak,
                          "frac": tf_dom / fp64_peak,
                          "peak_source": "FP64 FMA chains on every SM, measured in this run"},
            "kernels": {"aprod1": {"ms": t_a1 * 1e3, "GB/s": gbs_a1, "hbm_frac": gbs_a1 / hbm,
                                   "fp64_TFLOP/s": tf_a1, "fp64_frac": tf_a1 / fp64_peak,
                                   "split_products": split1, "api_call_ms": api_a1 * 1e3},
                        "aprod2": {"ms": t_a2 * 1e3, "GB/s": gbs_a2, "hbm_frac": gbs_a2 / hbm,
                                   "fp64_TFLOP/s": tf_a2, "fp64_frac": tf_a2 / fp64_peak,
                                   "split_products": split2, "api_call_ms": api_a2 * 1e3},
                        "vector_pass": {"ms": t_vec * 1e3, "GB/s": bytes_vec / t_vec / 1e9,
                                        "hbm_frac": bytes_vec / t_vec / 1e9 / hbm}},
            "aprod_GB/s": (bytes_a1 + bytes_a2) / (t_a1 + t_a2) / 1e9,
            "aprod_hbm_frac": (bytes_a1 + bytes_a2) / (t_a1 + t_a2) / 1e9 / hbm}

    mixed = None
    batched = None
    large = {}
    if (not args.no_mixed or not args.no_batched) and rank == 0:
        with Solver(sys_, conlim=0.0, precision=_lib.GSR_PREC_MIXED) as sm:
            if not args.no_mixed:
                mixed = time_to_solution(sm, b, torch, stream)
            if not args.no_batched:
                batched = batched_vs_sequential(
                    sm, xt, lambda j: torch.tensor(gen.noise(sys_, seed + 1000 * (j + 1)), device=dev),
                    torch, stream)
    if rank == 0 and ws == 1 and not args.no_large:
        # the 1,000,000-star mixed-precision and 2,000,000-star batched
        # workloads, generated on the device once the medium handles are gone
        solver.close()
        torch.cuda.empty_cache()
        for name in ("large", "xlarge"):
            try:
                large[name] = large_comparison(name, torch, stream)
            except Exception as e:  # reported, never fatal for the main line
                large[name] = {"unavailable": ("%s: %s" % (type(e).__name__, e))[:300]}

    # per solve (ncu launch list of --eager): 8 prologue launches (2 clears,
    # preconditioner: single-launch aprod 2 of squares + combine + finish;
    # init: U, aprod 2, first vector pass), 3 per LSQR iteration (aprod 1,
    # single-launch aprod 2, vector pass that also combines aprod 2's
    # partial sums), 1 epilogue
    launches_per_step = 9 + 3 * (iters // args.steps)
    line = {"metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "stars": sys_.n_stars, "m": m, "n": n,
                       "n_dfa": sys_.n_dfa, "n_instr": sys_.n_instr, "itmax": itmax,
                       "iterations_per_step": iters / args.steps, "atol": 0.0, "btol": 0.0,
                       "l2": "inputs larger than L2 (%.2f GB matrix)" % (m * 208 / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": roof, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": launches_per_step * args.steps}
    if mixed is not None:
        line["mixed_vs_fp64"] = mixed
    if batched is not None:
        line["batched_vs_sequential_fp64"] = batched
    if "large" in large:
        line["large_mixed_vs_fp64"] = large["large"]
    if "xlarge" in large:
        line["xlarge_batched_vs_sequential_fp64"] = large["xlarge"]
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sys_, seed, args.cpu_seconds)
        try:
            line["cpu_baseline_openmp"] = cpu_baseline_openmp(sys_, seed, args.cpu_seconds)
        except OSError as e:  # library not built on this host
            line["cpu_baseline_openmp"] = {"unavailable": str(e)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
