"""Host-side planning of an index: the multi-level grid for a field and a set
of hit points, and a pair capacity that does not overflow.

The plan follows the data: the finest cell fits the small Gaussians (their
k-sigma box spans at most max_span cells), enough levels double the cell up
to the largest Gaussians, the query level is the level whose cell is closest
to `query_cell`, and the hash table has about one bucket per expected
(cell, Gaussian) entry.
Only the grid geometry is chosen here; every per-Gaussian and per-hit-point
computation runs in libgpf."""

from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import torch

from . import _abi
from .api import Field, GridConfig, Index, Queries

COORD_BITS = 20


def scene_bounds(field: Field, queries: Queries, pad: float = 1e-3):
    """Lower and upper corner of the Gaussian means and the valid hit points."""
    parts_lo, parts_hi = [], []
    if field.n:
        parts_lo.append(field.mean.amin(dim=1))
        parts_hi.append(field.mean.amax(dim=1))
    x = queries.x
    if queries.valid is not None and queries.m:
        x = x[:, queries.valid.bool()]
    if x.shape[1]:
        parts_lo.append(x.amin(dim=1))
        parts_hi.append(x.amax(dim=1))
    if not parts_lo:
        return [0.0, 0.0, 0.0], [1.0, 1.0, 1.0]
    lo = torch.stack(parts_lo).amin(dim=0).cpu().tolist()
    hi = torch.stack(parts_hi).amax(dim=0).cpu().tolist()
    return [v - pad for v in lo], [v + pad for v in hi]


def plan_grid(field: Field, queries: Queries, cutoff_sigma: float = 3.0, max_span: int = 4,
              query_cell: Optional[float] = None, hash_bits: Optional[int] = None,
              bounds: Optional[Sequence] = None, small_quantile: float = 0.01,
              brute_force: bool = False) -> GridConfig:
    """Grid geometry for (field, queries); capacities are left at 0."""
    lo, hi = bounds if bounds is not None else scene_bounds(field, queries)
    ext = max(max(h - l for l, h in zip(lo, hi)), 1e-6)
    k = 3.0 if math.isinf(cutoff_sigma) else cutoff_sigma
    if field.n:
        # conservative half-extent of every Gaussian's k-sigma box: k * max scale
        e = k * torch.exp(field.logscale.amax(dim=0).double())
        e_small = float(torch.quantile(e[: 1 << 24], small_quantile)) if field.n > 1 else float(e[0])
        e_large = float(e.max())
    else:
        e_small = e_large = ext / 64
    span = max(1, max_span - 1)
    c_min = ext / (1 << COORD_BITS) * 4.0
    c0 = max(2.0 * e_small / span, c_min)
    top = max(2.0 * e_large / span, c0)
    levels = int(min(_abi.GPF_MAX_LEVELS, max(1, math.ceil(math.log2(top / c0)) + 1)))
    if query_cell is None:
        query_cell = ext / 256.0
    best = None
    for K in range(0, 16):
        cq = c0 * (1 << K)
        dims = [max(1, int(math.ceil((h - l) / cq))) for l, h in zip(lo, hi)]
        if any(d > _abi.GPF_MAX_DIM for d in dims) or any(d << K > (1 << COORD_BITS) for d in dims):
            continue
        if dims[0] * dims[1] * dims[2] > (1 << 26):
            continue
        score = abs(math.log2(cq / query_cell))
        if best is None or score < best[0]:
            best = (score, K, dims)
    if best is None:            # coarsen the finest cell until a query level fits
        c0 = ext / _abi.GPF_MAX_DIM * 1.001
        best = (0.0, 0, [max(1, int(math.ceil((h - l) / c0))) for l, h in zip(lo, hi)])
        levels = max(1, min(_abi.GPF_MAX_LEVELS,
                            int(math.ceil(math.log2(max(top / c0, 1.0)))) + 1))
    _, K, dims = best
    if hash_bits is None:
        # about one bucket per expected (cell, Gaussian) entry (~16 per Gaussian)
        want = max(16 * max(field.n, 1), 4 * max(queries.m, 1))
        hash_bits = int(min(26, max(12, math.ceil(math.log2(want)))))
    return GridConfig(list(lo), c0, levels, max_span, K, dims, hash_bits, field.channels,
                      cutoff_sigma, 0, 0, 0, brute_force)


def make_index(field: Field, queries: Queries, cutoff_sigma: float = 3.0,
               brute_force: bool = False, max_pairs: Optional[int] = None,
               bounds: Optional[Sequence] = None, max_gaussians: Optional[int] = None,
               max_queries: Optional[int] = None, headroom: float = 1.1, max_span: int = 4,
               query_cell: Optional[float] = None, hash_bits: Optional[int] = None,
               grid: Optional[GridConfig] = None, coop_cells: int = 0,
               ball_radius: Optional[float] = None, max_nb_pairs: int = 0,
               split_items: Optional[int] = None) -> Index:
    """An index planned for (field, queries). With max_pairs=None the pair
    capacity comes from a trial build (gpf_index_stats) times `headroom`
    (room for the pairs to grow while the parameters are optimised)."""
    if grid is None:
        # plan on the float32 values (a GPF_BF16 field is decoded for this)
        grid = plan_grid(field.decoded(), queries, cutoff_sigma, max_span, query_cell, hash_bits,
                         bounds, brute_force=brute_force)
        grid.coop_cells = coop_cells
    else:
        grid = dataclasses.replace(grid)     # capacities below are this index's own
    grid.field_storage = field.storage
    if ball_radius is not None:
        grid.ball_radius = float(ball_radius)
    grid.max_nb_pairs = int(max_nb_pairs)
    if split_items is not None:
        grid.split_items = int(split_items)
    grid.max_gaussians = max_gaussians if max_gaussians is not None else max(field.n, 1)
    grid.max_queries = max_queries if max_queries is not None else max(queries.m, 1)
    brute = brute_force or math.isinf(cutoff_sigma)
    grid.brute_force = brute_force
    grid.max_pairs = 1 if brute else (max_pairs if max_pairs is not None
                                      else max(8 * grid.max_gaussians, 1024))
    idx = Index(grid, device=field.mean.device)
    if brute or max_pairs is not None:
        return idx
    idx.build(field, queries)
    st = idx.stats()
    want = int(st["n_pairs"] * headroom) + 1024
    if st["overflow"] or want > grid.max_pairs:
        grid.max_pairs = want
        idx = Index(grid, device=field.mean.device)
    return idx


def time_step(index: Index, field: Field, queries: Queries, mode: int = 0, r_max: float = 0.02,
              repeats: int = 3, backward: bool = True) -> float:
    """Fastest of `repeats` runs of build + forward (+ backward) with `index`,
    in milliseconds (the fastest run is the one least disturbed by other work
    on the GPU or host)."""
    from . import api
    out = torch.empty((field.channels, queries.m), device=field.mean.device)
    z = torch.empty((queries.m,), device=field.mean.device)
    gout = torch.ones_like(out)
    grads = Field.zeros_like(field)
    times = []
    for i in range(repeats + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        index.build(field, queries)
        api.gpf_radiance_fwd(index, field, queries, mode, r_max=r_max, out=out, z=z)
        if backward:
            api.gpf_radiance_bwd(index, field, queries, gout, out, z, mode, r_max=r_max,
                                 grads=grads)
        e1.record()
        e1.synchronize()
        if i:                       # the first run pays one-off costs
            times.append(e0.elapsed_time(e1))
    return float(min(times))


def autotune(field: Field, queries: Queries, cutoff_sigma: float = 3.0, mode: int = 0,
             r_max: float = 0.02, query_cells: Optional[Sequence[float]] = None,
             max_spans: Sequence[int] = (3, 4, 6), coop_options: Sequence[int] = (2, 4, 8),
             repeats: int = 3, headroom: float = 1.25, backward: bool = True,
             split_options: Sequence[int] = (0, 4096, 16384)):
    """Chooses the grid geometry and the forward tile shape for this field
    and batch of hit points by timing build + forward + backward, one knob at
    a time: the query cell size (the hit-point grid), then the largest span of
    a Gaussian's box in cells of its level (the cell size of every level),
    then the cooperative-mode threshold of the forward's 32-point tiles,
    then the work above which a tile is split over several units (0: never),
    and last the query cell again with the other knobs settled. Each trial
    scores the fastest of `repeats` runs. Returns (best GridConfig, report), report = [(knobs, ms), ...] in the
    order tried. Results are independent of the choice; only speed differs.
    backward=False times build + forward only (a query without gradient,
    such as the GPF_DISK_KDE gather)."""
    if query_cells is None:
        query_cells = (0.01, 0.02, 0.04, 0.08)
    best = {"query_cell": 0.02, "max_span": 4, "coop_cells": 4,
            "split_items": split_options[0]}    # the first option while the others are tuned
    report = []
    cache = {}

    def trial(knobs):
        key = tuple(sorted(knobs.items()))
        if key not in cache:
            idx = make_index(field, queries, cutoff_sigma=cutoff_sigma, headroom=headroom,
                             query_cell=knobs["query_cell"], max_span=knobs["max_span"],
                             coop_cells=knobs["coop_cells"], split_items=knobs["split_items"])
            ms = time_step(idx, field, queries, mode, r_max, repeats, backward)
            cache[key] = (ms, idx.grid)
            report.append((dict(knobs), ms))
            del idx
            torch.cuda.empty_cache()
        return cache[key][0]

    # one knob at a time, then the query cell once more with the others
    # settled (its first pass saw their initial values)
    for name, options in (("query_cell", query_cells), ("max_span", max_spans),
                          ("coop_cells", coop_options), ("split_items", split_options),
                          ("query_cell", query_cells)):
        scores = {}
        for v in options:
            knobs = dict(best, **{name: v})
            scores[v] = trial(knobs)
        best[name] = min(scores, key=lambda v: (scores[v], v))
    grid = cache[tuple(sorted(best.items()))][1]
    return grid, report
