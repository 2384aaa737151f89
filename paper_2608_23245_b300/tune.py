"""Autotuner of the batched refinement step's launch shapes.

Times fdx_batch_refine on the caller's own models for a small grid of
fdx_tuning settings (pixels per lane, persistent CTAs per SM of the forward
and adjoint kernels, adjoint bands per reflection), keeps the fastest, sets it
process-wide, and caches the choice in a JSON file keyed by a signature of
the workload (model count, detector sizes, reflection and atom counts, node
grids), so a later run of the same workload starts from the tuned setting.
All timing is on the device with CUDA events.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

from . import fdx

DEFAULT_GRID = {
    "ppl_max": (2, 1),
    "fwd_ctas_per_sm": (4, 3),
    "adj_ctas_per_sm": (3, 2),
    "adj_bands": (64, 32, 128),
}


def signature(problems, datoms) -> str:
    key = [(p.geom.n_x, p.geom.n_y, p.n_refl, p.br.n_nodes, int(d.frac.shape[0])) for p, d in zip(problems, datoms)]
    return hashlib.sha1(json.dumps(key).encode()).hexdigest()[:16]


def _time_step(problems, datoms, targets, reps):
    import torch
    step = fdx.BatchStep(problems, datoms, targets=targets)
    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        step()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune_batch(problems, datoms, targets, grid=None, reps=1, cache_path=None, verbose=False):
    """Return (best tuning dict, {setting: ms}) and apply the best setting."""
    grid = grid or DEFAULT_GRID
    sig = signature(problems, datoms)
    if cache_path and os.path.exists(cache_path):
        try:
            cached = json.load(open(cache_path)).get(sig)
        except (OSError, ValueError):
            cached = None
        if cached:
            fdx.fdx_set_tuning(fdx.Tuning(**cached["best"]))
            return cached["best"], cached["timings"]
    names = list(grid)
    timings = {}
    best, best_ms = None, float("inf")
    for combo in itertools.product(*(grid[k] for k in names)):
        t = dict(zip(names, combo))
        fdx.fdx_set_tuning(fdx.Tuning(**t))
        ms = _time_step(problems, datoms, targets, reps)
        timings[json.dumps(t, sort_keys=True)] = ms
        if verbose:
            print("tune", t, "%.2f ms" % ms, flush=True)
        if ms < best_ms:
            best, best_ms = t, ms
    fdx.fdx_set_tuning(fdx.Tuning(**best))
    if cache_path:
        data = {}
        if os.path.exists(cache_path):
            try:
                data = json.load(open(cache_path))
            except (OSError, ValueError):
                data = {}
        data[sig] = {"best": best, "timings": timings}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        json.dump(data, open(cache_path, "w"), indent=1, sort_keys=True)
    return best, timings
