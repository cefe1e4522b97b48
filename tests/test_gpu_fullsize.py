"""Parity at the benchmark's full size and grid: 1,000,000 Gaussians of the
caustic floor + sphere scene, one 1024 x 1024 view (728,666 active hit
points), 3-sigma truncation, r = 0.02, the grid the benchmark profiles
(query cell 0.0308, max span 3, cooperative tiles up to 8 cells), one
training step's forward, MSE gradient against the perturbed target, and
backward (Sec. 4.2 aggregation equation and Differentiable Accumulation).

The oracle cannot sum a million Gaussians for every hit point in a test,
so each check restricts its inputs by a condition the definition implies:
  * forward: at a sampled hit point x only Gaussians with |x - mu| <= 3 s_max
    can have Q <= 9 (Q = |S^-1 R^T d|^2 >= |d|^2 / s_max^2), so the oracle
    gets every Gaussian whose sphere of that radius (x 1.001) reaches a
    sampled point, and the rest of the field would add exact zeros;
  * backward, GPF_SUM: the gradient of Gaussian i is a sum over its own pairs
    (i, x) weighted by the upstream gradient at x, independent of every other
    Gaussian, so the oracle gets the chosen Gaussians alone and the hit
    points their spheres reach.
The sampled hit points include every point of the 32 tiles (32 consecutive
points in the library's cell order) whose points have the most Gaussian
means nearby, which is where the forward's pooled mode walks its longest
lists, and so also the points at those tiles' boundaries. The chosen
Gaussians include the 64 largest, among them the ones the backward splits
into several work units, and the test asserts that the build split some."""

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import FWD_TOL, GRAD_TOL, fwd_rel_err

pytestmark = pytest.mark.gpu

R = 0.02
KEYS = ("mean", "quat", "logscale", "spectrum")


@pytest.fixture(scope="module")
def scene():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pytest.importorskip("scipy")
    import paper_2512_12459_gb300 as gpf
    from paper_2512_12459_gb300.setup_index import make_index
    pos, flux = synth.caustic_photons(1_000_000, seed=0)
    fnp = synth.field_from_photons(pos, flux, seed=0)
    tnp = synth.perturbed_copy(fnp, seed=1)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 1024, 1024)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    tf = gpf.Field.from_numpy(tnp)
    tidx = make_index(tf, queries, query_cell=0.02)
    tidx.build(tf, queries)
    target = gpf.gpf_radiance_fwd(tidx, tf, queries, gpf.GPF_SUM, r_max=R)[0].clone()
    del tidx, tf
    return {"gpf": gpf, "fnp": fnp, "qnp": qnp, "field": field, "queries": queries,
            "target": target, "runs": {}}


def _run(scene, query_cell):
    """One step's forward, MSE gradient and backward on the grid of this query
    cell (max span 3, cooperative tiles up to 8 cells)."""
    if query_cell in scene["runs"]:
        return scene["runs"][query_cell]
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    gpf, field, queries = scene["gpf"], scene["field"], scene["queries"]
    idx = make_index(field, queries, cutoff_sigma=3.0, headroom=1.25, query_cell=query_cell,
                     max_span=3, coop_cells=8)
    idx.build(field, queries)
    out, z = gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=R)
    _, gout = gpf.gpf_mse_loss_grad(out, scene["target"], queries.valid)
    grads = gpf.gpf_radiance_bwd(idx, field, queries, gout, out, z, gpf.GPF_SUM, r_max=R)
    torch.cuda.synchronize()
    r = {"grid": idx.grid, "stats": idx.stats(raise_on_flags=True),
         "out": out.cpu().numpy().astype(np.float64),
         "gout": gout.cpu().numpy().astype(np.float64),
         "grads": {k: getattr(grads, k).cpu().numpy().astype(np.float64) for k in KEYS}}
    scene["runs"][query_cell] = r
    del idx
    return r


def _cell_keys(grid, x):
    """Query-level cell keys of points x [3, n] (float32 cell coordinates as
    the build computes them)."""
    f32 = np.float32
    K = grid.query_level
    inv = f32(1.0) / f32(grid.cell_size)
    c = []
    for a in range(3):
        t = np.floor((x[a].astype(f32) - f32(grid.origin[a])) * inv)
        cmax = (grid.dims[a] << K) - 1
        c.append(np.clip(t, 0, cmax).astype(np.int64) >> K)
    return (c[2] * grid.dims[1] + c[1]) * grid.dims[0] + c[0]


def _sorted_order(grid, qnp):
    """Hit points in the library's tile order: stable sort by the query-level
    cell key, inactive points last."""
    key = _cell_keys(grid, qnp.x)
    active = qnp.valid.astype(bool) & (np.sum(qnp.n.astype(np.float64) * qnp.wo, axis=0) > 0)
    key[~active] = grid.dims[0] * grid.dims[1] * grid.dims[2]
    return np.argsort(key, kind="stable"), active


def _sphere_radius(fnp):
    return 3.0 * np.exp(fnp.logscale.astype(np.float64).max(axis=0)) * 1.001


def test_full_size_forward_heaviest_tiles(scene):
    from scipy.spatial import cKDTree
    run = _run(scene, 0.0308)
    fnp, qnp, grid = scene["fnp"], scene["qnp"], run["grid"]
    order, active = _sorted_order(grid, qnp)
    n_act = int(active.sum())
    assert n_act == run["stats"]["n_active"]
    tiles = order[: (n_act // 32) * 32].reshape(-1, 32)
    means = fnp.mean.T.astype(np.float64)
    # weight of a tile: the Gaussian means in its points' query-level cells
    # (the forward's list items grow with the density of Gaussians there)
    qkey = _cell_keys(grid, qnp.x)
    mkey = _cell_keys(grid, fnp.mean)
    cells, counts = np.unique(mkey, return_counts=True)
    pos = np.clip(np.searchsorted(cells, qkey), 0, cells.size - 1)
    dens = np.where(cells[pos] == qkey, counts[pos], 0)
    weight = dens[tiles].sum(axis=1)
    heavy = tiles[np.argsort(-weight, kind="stable")[:32]].ravel()
    rng = np.random.default_rng(11)
    rand = rng.choice(np.flatnonzero(active), size=256, replace=False)
    tail = order[max(0, n_act - 37):n_act]            # the ragged last tile
    sel = np.unique(np.concatenate([heavy, rand, tail]))
    assert sel.size >= 256 + 32 * 16
    # every Gaussian whose bounding sphere reaches a sampled point
    reach = cKDTree(qnp.x.T[sel].astype(np.float64)).query_ball_point(
        means, r=_sphere_radius(fnp), return_length=True, workers=-1)
    sub = synth.subset_field(fnp, np.flatnonzero(reach > 0))
    q = synth.subset_queries(qnp, sel)
    ref = oracle.radiance_fwd(sub.mean, sub.quat, sub.logscale, sub.spectrum, q.x, q.n, q.wo,
                              None, q.valid, mode=oracle.GPF_SUM, r_max=R, cutoff_sigma=3.0)
    err, zero_ok = fwd_rel_err(run["out"][:, sel], ref)
    assert zero_ok and err < FWD_TOL, err
    # the heavy tiles lie where the Gaussians are densest (and so smallest)
    heavy_pos = np.isin(sel, heavy)
    assert dens[sel[heavy_pos]].mean() > 4.0 * dens[sel[~heavy_pos]].mean()
    assert ref["near_cutoff"].sum() < 0.05 * sel.size


def _query_boxes(grid, fnp, gsel):
    """Query-level cell count of the k-sigma bounds of the chosen Gaussians
    (the build's size classes, in float64: a check of the test's choice)."""
    from oracle.gpf_oracle import quat_to_rotmat
    q = fnp.quat[:, gsel].T.astype(np.float64)
    R_ = quat_to_rotmat(q / np.linalg.norm(q, axis=1, keepdims=True))
    s = np.exp(fnp.logscale[:, gsel].T.astype(np.float64))
    e = 3.0 * np.sqrt(np.einsum("nkj,nj->nk", R_ ** 2, s ** 2))
    mu = fnp.mean[:, gsel].T.astype(np.float64)
    cq = grid.cell_size * (1 << grid.query_level)
    o = np.asarray(grid.origin, dtype=np.float64)
    lo = np.floor((mu - e - o) / cq)
    hi = np.floor((mu + e - o) / cq)
    dims = np.asarray(grid.dims)
    lo, hi = np.clip(lo, 0, dims - 1), np.clip(hi, 0, dims - 1)
    return np.prod(hi - lo + 1, axis=1)


@pytest.mark.parametrize("query_cell", [0.0308, 0.0154])
def test_full_size_backward_subset(scene, query_cell):
    """The benchmark's grid (query cell 0.0308: no Gaussian's bounds reach 2^12
    query cells, so nothing is split) and the next finer query level (0.0154,
    where the largest Gaussians are split into GPF_BWD_SPLIT_WAYS units)."""
    from scipy.spatial import cKDTree
    run = _run(scene, query_cell)
    fnp, qnp, grid, st = scene["fnp"], scene["qnp"], run["grid"], run["stats"]
    assert st["n_small"] > 0 and st["n_live"] > st["n_small"]
    rng = np.random.default_rng(12)
    smax = np.exp(fnp.logscale.astype(np.float64).max(axis=0))
    largest = np.argsort(-smax, kind="stable")[:64]
    gsel = np.unique(np.concatenate([largest, rng.choice(fnp.n, size=512, replace=False)]))
    # the chosen Gaussians cover the backward's classes: small ones (a lane
    # each) and, on the finer grid, split ones (bounds over 2^12 query cells)
    vq = _query_boxes(grid, fnp, gsel)
    assert (vq <= 8).sum() >= 100, vq.min()
    if query_cell < 0.02:
        assert st["n_huge"] > 0 and st["n_split"] == min(st["n_huge"], 16384)
        assert (vq >= 4096 * 1.5).sum() >= 1, vq.max()
    active = qnp.valid.astype(bool) & (np.sum(qnp.n.astype(np.float64) * qnp.wo, axis=0) > 0)
    act = np.flatnonzero(active)
    tree = cKDTree(qnp.x.T[act].astype(np.float64))
    lists = tree.query_ball_point(fnp.mean.T[gsel].astype(np.float64),
                                  r=_sphere_radius(fnp)[gsel], workers=-1)
    pts = act[np.unique(np.concatenate([np.asarray(l, dtype=np.int64) for l in lists]))]
    sub = synth.subset_field(fnp, gsel)
    q = synth.subset_queries(qnp, pts)
    ref = oracle.radiance_bwd(sub.mean, sub.quat, sub.logscale, sub.spectrum, q.x, q.n, q.wo,
                              run["gout"][:, pts], None, q.valid, mode=oracle.GPF_SUM, r_max=R,
                              cutoff_sigma=3.0)
    # The field's Gaussians are isotropic (one scale per photon), so the
    # exact quaternion gradient is zero and float32 leaves rounding noise of
    # the size of the sums A that also give the log-scale gradient: the
    # quaternion errors are measured against |d quat| + |d logscale|.
    worst, norm = {}, {}
    for k in KEYS:
        g, r = run["grads"][k][:, gsel], ref[k]
        extra = ref["logscale"] if k == "quat" else np.zeros_like(r)
        norm[k] = float(np.linalg.norm(g - r) / (np.linalg.norm(r) + np.linalg.norm(extra)))
        # per Gaussian: within 1e-3 of its own gradient or of the RMS over the chosen ones
        own = np.linalg.norm(r, axis=0) + np.linalg.norm(extra, axis=0)
        scale = own + (np.linalg.norm(r) + np.linalg.norm(extra)) / np.sqrt(gsel.size)
        per = np.linalg.norm(g - r, axis=0) / scale
        worst[k] = float(per.max())
    for k in KEYS:
        assert norm[k] < GRAD_TOL, (k, norm)
        assert worst[k] < 1e-3, (k, worst)
    print(f"full-size backward (query cell {query_cell}, {st['n_split']} split, "
          f"{int((vq >= 4096).sum())} of the chosen over 2^12 cells): normwise {norm}, "
          f"per-Gaussian worst {worst}")
