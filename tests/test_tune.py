"""Host logic of the autotuner (paper_2608_23245_b300/tune.py): the search
over fdx_tuning settings, complete settings built from the library defaults,
and the JSON cache keyed by the workload signature.  The timing of a step is
replaced by a synthetic cost, so no GPU is needed."""
import json
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2608_23245_b300 import fdx, tune


def _fake(monkeypatch, cost):
    """Route fdx_set_tuning and the step timer to a synthetic cost of the
    current setting; returns the list of settings applied."""
    applied = []
    state = {}

    def set_tuning(t=None):
        d = t.as_dict()
        for k in ("ppl_max", "fwd_ctas_per_sm", "adj_ctas_per_sm", "adj_bands", "node_block"):
            assert k in d
        assert 1 <= d["ppl_max"] <= 2 and 1 <= d["fwd_ctas_per_sm"] <= 8 and 1 <= d["adj_ctas_per_sm"] <= 8
        assert 1 <= d["adj_bands"] <= 256 and 0 <= d["node_block"] <= 3
        state["t"] = d
        applied.append(d)

    monkeypatch.setattr(fdx, "fdx_set_tuning", set_tuning)
    monkeypatch.setattr(tune, "_time_step", lambda problems, datoms, targets, reps: cost(state["t"]))
    return applied


def _workload(n=3):
    probs = [SimpleNamespace(geom=SimpleNamespace(n_x=64 + k, n_y=32), n_refl=100 + k, br=SimpleNamespace(n_nodes=16))
             for k in range(n)]
    atoms = [SimpleNamespace(frac=np.zeros((10 + k, 3))) for k in range(n)]
    return probs, atoms


def _separable(t):
    return (1.0 * (t["ppl_max"] != 1) + 2.0 * abs(t["node_block"] - 2) + 0.5 * abs(t["fwd_ctas_per_sm"] - 3)
            + 0.25 * abs(t["adj_ctas_per_sm"] - 2) + 0.01 * abs(t["adj_bands"] - 32))


def test_coordinate_search_finds_separable_optimum(monkeypatch):
    applied = _fake(monkeypatch, _separable)
    probs, atoms = _workload()
    best, timings = tune.autotune_batch(probs, atoms, [None] * 3)
    assert best == {"ppl_max": 1, "node_block": 2, "fwd_ctas_per_sm": 3, "adj_ctas_per_sm": 2, "adj_bands": 32}
    # one timing per distinct setting: 1 + (2-1) + (4-1) + (2-1) + (2-1) + (3-1)
    assert len(timings) == 1 + sum(len(v) - 1 for v in tune.DEFAULT_GRID.values())
    assert applied[-1] == best  # the best setting is left applied


def test_coordinate_search_starts_from_defaults(monkeypatch):
    applied = _fake(monkeypatch, _separable)
    probs, atoms = _workload()
    tune.autotune_batch(probs, atoms, [None] * 3, grid={"node_block": (1, 2)})
    for d in applied:
        for k, v in fdx.Tuning.DEFAULTS.items():
            if k != "node_block":
                assert d[k] == v
    assert applied[-1]["node_block"] == 2


def test_grid_search_finds_global_optimum(monkeypatch):
    # a coupled cost whose coordinate-wise optimum from the defaults is not the global one
    def coupled(t):
        return 0.0 if (t["ppl_max"] == 1 and t["node_block"] == 3) else (1.0 if t["ppl_max"] == 2 else 2.0)
    _fake(monkeypatch, coupled)
    probs, atoms = _workload()
    grid = {"ppl_max": (2, 1), "node_block": (0, 3)}
    best_c, _ = tune.autotune_batch(probs, atoms, [None] * 3, grid=grid)
    assert best_c["ppl_max"] == 2
    best_g, timings = tune.autotune_batch(probs, atoms, [None] * 3, grid=grid, method="grid")
    assert best_g["ppl_max"] == 1 and best_g["node_block"] == 3
    assert len(timings) == 4
    with pytest.raises(ValueError):
        tune.autotune_batch(probs, atoms, [None] * 3, grid=grid, method="random")


def test_cache_round_trip(monkeypatch, tmp_path):
    applied = _fake(monkeypatch, _separable)
    probs, atoms = _workload()
    path = str(tmp_path / "sub" / "tune.json")
    best, timings = tune.autotune_batch(probs, atoms, [None] * 3, cache_path=path)
    data = json.load(open(path))
    sig = tune.signature(probs, atoms)
    assert data[sig]["best"] == best
    n = len(applied)
    best2, timings2 = tune.autotune_batch(probs, atoms, [None] * 3, cache_path=path)
    assert best2 == best and timings2 == timings
    assert len(applied) == n + 1 and applied[-1] == best  # applied from the cache, nothing timed
    # another workload gets its own entry
    probs3, atoms3 = _workload(4)
    tune.autotune_batch(probs3, atoms3, [None] * 4, cache_path=path)
    assert len(json.load(open(path))) == 2


def test_tuning_struct_defaults():
    t = fdx.Tuning.of(node_block=1)
    d = t.as_dict()
    assert d["node_block"] == 1 and d["ppl_max"] == 2 and d["adj_bands"] == 128
    assert set(d) == set(fdx.Tuning.DEFAULTS)
