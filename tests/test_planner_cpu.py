"""The host-side grid planner (setup_index.plan_grid) on CPU tensors: the
geometry it hands to gpf_index_create respects the library's limits, puts
the largest Gaussians within the span bound on the top level and the small
ones on level 0, and picks the query level nearest the asked cell size."""

import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

from paper_2512_12459_gb300 import _abi  # noqa: E402
from paper_2512_12459_gb300.api import Field, Queries  # noqa: E402
from paper_2512_12459_gb300.setup_index import COORD_BITS, plan_grid, scene_bounds  # noqa: E402


def _scene(n=20000, seed=5):
    pos, flux = synth.caustic_photons(n, seed=seed)
    fnp = synth.field_from_photons(pos, flux, seed=seed)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 96, 80)
    t = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a), dtype=dt)  # noqa: E731
    field = Field(t(fnp.mean), t(fnp.quat), t(fnp.logscale), t(fnp.spectrum))
    queries = Queries(t(qnp.x), t(qnp.n), t(qnp.wo), None, t(qnp.valid, torch.uint8))
    return fnp, qnp, field, queries


@pytest.mark.parametrize("max_span", [3, 4, 6])
@pytest.mark.parametrize("query_cell", [0.01, 0.03, 0.08])
def test_plan_respects_limits_and_spans(max_span, query_cell):
    fnp, qnp, field, queries = _scene()
    g = plan_grid(field, queries, cutoff_sigma=3.0, max_span=max_span, query_cell=query_cell)
    assert 1 <= g.levels <= _abi.GPF_MAX_LEVELS
    assert 0 <= g.query_level <= 15 and 12 <= g.hash_bits <= 26
    for d in g.dims:
        assert 1 <= d <= _abi.GPF_MAX_DIM
        assert d << g.query_level <= 1 << COORD_BITS
    c0 = g.cell_size
    # the k-sigma half-extent bound of every Gaussian: k * max scale
    e = 3.0 * np.exp(fnp.logscale.astype(np.float64).max(axis=0))
    span = max_span - 1
    assert 2.0 * e.max() <= span * c0 * 2 ** (g.levels - 1) * (1 + 1e-9)
    if c0 > 0 and g.levels < _abi.GPF_MAX_LEVELS:
        # one level fewer would not hold the largest Gaussian within the span
        assert g.levels == 1 or 2.0 * e.max() > span * c0 * 2 ** (g.levels - 2)
    # the query level is the one whose cell is nearest the asked size (in
    # log2) among the levels whose grid fits: at most GPF_MAX_DIM cells per
    # axis, 2^26 cells in all, and 2^20 finest cells per axis
    lo, hi = scene_bounds(field, queries)
    cq = c0 * 2 ** g.query_level

    def fits(k):
        c = c0 * 2 ** k
        dims = [max(1, math.ceil((h - l) / c)) for l, h in zip(lo, hi)]
        return (all(d <= _abi.GPF_MAX_DIM and d << k <= 1 << COORD_BITS for d in dims)
                and dims[0] * dims[1] * dims[2] <= 1 << 26)

    assert fits(g.query_level)
    for k in range(16):
        if k != g.query_level and fits(k):
            assert abs(math.log2(cq / query_cell)) <= \
                abs(math.log2(c0 * 2 ** k / query_cell)) + 1e-9


def test_scene_bounds_cover_means_and_valid_hit_points():
    fnp, qnp, field, queries = _scene(n=5000, seed=9)
    lo, hi = scene_bounds(field, queries)
    v = qnp.valid.astype(bool)
    for k in range(3):
        assert lo[k] < fnp.mean[k].min() and hi[k] > fnp.mean[k].max()
        assert lo[k] < qnp.x[k, v].min() and hi[k] > qnp.x[k, v].max()


def test_plan_of_an_empty_field_still_gives_a_grid():
    _, _, field, queries = _scene(n=2000, seed=3)
    empty = Field(*(t[:, :0].contiguous() for t in (field.mean, field.quat, field.logscale,
                                                    field.spectrum)))
    g = plan_grid(empty, queries, cutoff_sigma=3.0, max_span=3, query_cell=0.05)
    assert g.levels >= 1 and all(1 <= d <= _abi.GPF_MAX_DIM for d in g.dims)


def test_planned_grid_keeps_index_order_and_the_struct_carries_tile_order():
    """The planner leaves hit points in index order inside their cells
    (tile_order 0: the sub-cell order costs a fourth sort pass for a
    smaller gain in the forward on the benchmark scene), and the ctypes
    struct passes an explicit order through to gpf_index_create."""
    import dataclasses
    fnp, qnp, field, queries = _scene()
    g = plan_grid(field, queries, cutoff_sigma=3.0, query_cell=0.03)
    assert g.tile_order == 0 and g.c_struct().tile_order == 0
    g2 = dataclasses.replace(g, tile_order=min(2, g.query_level))
    assert g2.c_struct().tile_order == min(2, g.query_level)


def test_autotune_search_order_and_choice(monkeypatch):
    """The autotuner's search on a synthetic cost (no GPU): one knob at a
    time in the documented order, then the query cell again with the other
    knobs settled; every distinct setting is timed once; the result is the
    cheapest setting it visited."""
    from paper_2512_12459_gb300 import setup_index

    def cost(k):
        # the best query cell depends on the span, so the second pass matters
        best_cell = 0.02 if k["max_span"] == 3 else 0.04
        return (abs(math.log2(k["query_cell"] / best_cell)) + 2.0 * (k["max_span"] != 3)
                + 0.1 * (k["coop_cells"] != 8) + 0.05 * (k["split_items"] != 4096))

    class _Idx:
        def __init__(self, knobs):
            self.grid = dict(knobs)

    calls = []

    def fake_make_index(field, queries, cutoff_sigma=3.0, headroom=1.25, query_cell=None,
                        max_span=4, coop_cells=0, split_items=None, **kw):
        return _Idx(dict(query_cell=query_cell, max_span=max_span, coop_cells=coop_cells,
                         split_items=split_items))

    def fake_time_step(index, field, queries, mode, r_max, repeats, backward):
        calls.append(dict(index.grid))
        return cost(index.grid)

    monkeypatch.setattr(setup_index, "make_index", fake_make_index)
    monkeypatch.setattr(setup_index, "time_step", fake_time_step)
    grid, report = setup_index.autotune(None, None, query_cells=(0.01, 0.02, 0.04),
                                        max_spans=(3, 4), coop_options=(4, 8),
                                        split_options=(0, 4096))
    assert grid == {"query_cell": 0.02, "max_span": 3, "coop_cells": 8, "split_items": 4096}
    # each distinct setting timed once, in the order reported
    keys = [tuple(sorted(c.items())) for c in calls]
    assert len(keys) == len(set(keys)) == len(report)
    assert [k for k, _ in report] == calls
    # first the query cell (3 settings, at the initial span 4: 0.04 wins),
    # then span, coop, split, then the cell again (at span 3: 0.02 wins)
    assert [c["query_cell"] for c in calls[:3]] == [0.01, 0.02, 0.04]
    assert all(c["max_span"] == 4 for c in calls[:3])
    assert calls[3]["query_cell"] == 0.04
    assert min(ms for _, ms in report) == cost(grid)
