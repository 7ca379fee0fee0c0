"""Autotuner of the batched kernels.

Times the batched products (A32 X and A32^T Y on k columns) for every column
tile (1, 2, 4, 8) and lanes per star (8, 16, 32) on the caller's system and
keeps the fastest, cached per (shape, k, device) in a JSON file.  Timing uses
CUDA events on the solver's stream; the choice is applied with
Solver.set_batch_tiling.
"""
from __future__ import annotations

import json
import os

TILES = (1, 2, 4, 8)
LANES = (8, 16, 32)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "batch_tuning.json")


def _key(solver, k, device_name):
    return "S%d_D%d_I%d_m%d_k%d_%s" % (solver.n_stars, solver.n_dfa, solver.n_instr, solver.m, k,
                                        device_name.replace(" ", "_"))


def tune(solver, k, reps=3, cache=DEFAULT_CACHE, force=False):
    """Pick (kt, lanes) for k columns on this solver; returns (kt, lanes, table)."""
    import torch
    dev = torch.cuda.get_device_name()
    key = _key(solver, k, dev)
    table = {}
    if cache and os.path.exists(cache) and not force:
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
        if key in table:
            kt, lanes = table[key]["kt"], table[key]["lanes"]
            solver.set_batch_tiling(kt, lanes)
            return kt, lanes, table[key]
    g = torch.Generator(device="cuda").manual_seed(1)
    X = torch.randn((k, solver.n), dtype=torch.float64, device="cuda", generator=g)
    Y = torch.randn((k, solver.m), dtype=torch.float64, device="cuda", generator=g)
    times = {}
    for kt in TILES:
        for lanes in LANES:
            solver.set_batch_tiling(kt, lanes)
            solver.batched_products(X, Y)  # warm-up (builds buffers)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                solver.batched_products(X, Y)
            e1.record()
            torch.cuda.synchronize()
            times["%d,%d" % (kt, lanes)] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    kt, lanes = (int(v) for v in best.split(","))
    solver.set_batch_tiling(kt, lanes)
    entry = {"kt": kt, "lanes": lanes, "ms": times}
    if cache:
        table[key] = entry
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return kt, lanes, entry
