"""Autotuner of the batched refinement step's launch and chunk shapes.

Times fdx_batch_refine on the caller's own models over fdx_tuning settings --
the detector tile (pixels per lane: 8 x 8 or 8 x 4 pixel patches), the
quadrature-node block that the kernels cull and stage as one unit (4 x 8,
8 x 4, 2 x 16 or 16 x 2 nodes), persistent CTAs per SM of the forward and
adjoint kernels and the adjoint's bands per reflection -- keeps the fastest,
sets it process-wide, and caches the choice in a JSON file keyed by a
signature of the workload (model count, detector sizes, reflection and atom
counts, node grids), so a later run of the same workload starts from the
tuned setting.  The search is coordinate-wise by default (one knob at a time,
in the grid's order, the others at their best so far, starting from the
library defaults; sum of the grid's lengths timings) or over the full product
of the grid.  All timing is on the device with CUDA events.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

from . import fdx

DEFAULT_GRID = {
    "ppl_max": (2, 1),
    "node_block": (1, 0, 2, 3),
    "fwd_ctas_per_sm": (4, 3),
    "adj_ctas_per_sm": (3, 2),
    "adj_bands": (128, 64, 32),
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


def _search(grid, measure, method):
    """Best setting of `grid` under `measure(setting dict) -> ms`; returns
    (best dict, {json setting: ms}).  Every setting is complete: the library
    defaults overridden by the grid's knobs."""
    names = list(grid)
    timings = {}

    def run(t):
        key = json.dumps(t, sort_keys=True)
        if key not in timings:
            timings[key] = measure(t)
        return timings[key]

    if method == "grid":
        best = min((dict(fdx.Tuning.DEFAULTS, **dict(zip(names, combo)))
                    for combo in itertools.product(*(grid[k] for k in names))), key=run)
        return best, timings
    if method != "coordinate":
        raise ValueError("method must be 'coordinate' or 'grid'")
    best = dict(fdx.Tuning.DEFAULTS)
    for name in names:
        best = min((dict(best, **{name: v}) for v in grid[name]), key=run)
    return best, timings


def autotune_batch(problems, datoms, targets, grid=None, reps=1, cache_path=None, verbose=False,
                   method="coordinate"):
    """Return (best tuning dict, {setting: ms}) and apply the best setting."""
    grid = grid or DEFAULT_GRID
    sig = signature(problems, datoms)
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cached = json.load(f).get(sig)
        except (OSError, ValueError):
            cached = None
        if cached:
            fdx.fdx_set_tuning(fdx.Tuning.of(**cached["best"]))
            return cached["best"], cached["timings"]

    def measure(t):
        fdx.fdx_set_tuning(fdx.Tuning.of(**t))
        ms = _time_step(problems, datoms, targets, reps)
        if verbose:
            print("tune", t, "%.2f ms" % ms, flush=True)
        return ms

    best, timings = _search(grid, measure, method)
    fdx.fdx_set_tuning(fdx.Tuning.of(**best))
    if cache_path:
        data = {}
        if os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    data = json.load(f)
            except (OSError, ValueError):
                data = {}
        data[sig] = {"best": best, "timings": timings}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    return best, timings
