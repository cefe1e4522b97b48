"""Batched multi-view steps: views of uneven size in one batch, the step as a
captured CUDA graph, the per-view baseline and the autotuner."""

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import FWD_TOL, fwd_rel_err, oracle_fwd, sample_active

pytestmark = pytest.mark.gpu

R = 0.02


@pytest.fixture(scope="module")
def gpf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12459_gb300 as g
    return g


def _scene(n_photons=30000, n_views=6, seed=41, sides=(24, 40, 56)):
    pos, flux = synth.caustic_photons(n_photons, seed=seed)
    fnp = synth.field_from_photons(pos, flux, seed=seed)
    qnp = synth.uneven_views(n_views, seed=seed, sides=sides)
    tgt = synth.perturbed_copy(fnp, seed=seed + 1)
    return fnp, qnp, tgt


def _target(gpf, tgt_np, queries):
    from paper_2512_12459_gb300.setup_index import make_index
    tf = gpf.Field.from_numpy(tgt_np)
    idx = make_index(tf, queries, query_cell=0.05)
    idx.build(tf, queries)
    out, _ = gpf.gpf_radiance_fwd(idx, tf, queries, gpf.GPF_SUM, r_max=R)
    return out.clone()


def test_batched_forward_matches_oracle_and_per_view(gpf):
    """One batch over all views equals the oracle, and equals each view run
    through its own index (different cells and order: within tolerance)."""
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp, _ = _scene()
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.05)
    idx.build(field, queries)
    out, _ = gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=R)
    out = out.cpu().numpy().astype(np.float64)
    sel = sample_active(qnp, 400, seed=42)
    ref = oracle_fwd(fnp, qnp, oracle.GPF_SUM, R, 3.0, sel)
    err, zero_ok = fwd_rel_err(out[:, sel], ref)
    assert err <= FWD_TOL and zero_ok
    offs = qnp.view_offsets
    assert len(offs) == 7 and len(set(np.diff(offs))) > 1          # uneven views
    for v in range(len(offs) - 1):
        sub = synth.subset_queries(qnp, np.arange(offs[v], offs[v + 1]))
        qv = gpf.Queries.from_numpy(sub)
        iv = make_index(field, qv, query_cell=0.05)
        iv.build(field, qv)
        ov, _ = gpf.gpf_radiance_fwd(iv, field, qv, gpf.GPF_SUM, r_max=R)
        a = ov.cpu().numpy().astype(np.float64)
        b = out[:, offs[v]:offs[v + 1]]
        scale = np.maximum(np.abs(b), 1e-30)
        assert np.all(np.abs(a - b) <= 2e-6 * scale + 1e-30)
    torch.cuda.synchronize()


def test_graph_replay_equals_eager_steps(gpf):
    """The captured step replays exactly what eager steps compute, Adam's
    update count advancing on the device."""
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    from paper_2512_12459_gb300.train import TrainStep
    fnp, qnp, tgt = _scene(seed=43)
    queries = gpf.Queries.from_numpy(qnp)
    target = _target(gpf, tgt, queries)
    fa, fb = gpf.Field.from_numpy(fnp), gpf.Field.from_numpy(fnp)
    ia = make_index(fa, queries, query_cell=0.05, headroom=1.5)
    ib = make_index(fb, queries, grid=ia.grid)
    sa = TrainStep(fa, queries, target, ia, r_max=R, lr=5e-3)
    sb = TrainStep(fb, queries, target, ib, r_max=R, lr=5e-3)
    sb.capture(warmup=1)                 # one real step, then the recording
    sa()                                 # the matching eager step
    losses = []
    for _ in range(6):
        sa()
        sb()
        torch.cuda.synchronize()
        losses.append((sa.loss_value(), sb.loss_value()))
    assert sa.updates() == 7 and sb.updates() == 7
    assert all(x == y for x, y in losses)
    assert losses[-1][0] < losses[0][0]                              # it trains
    for x, y in zip(fa.tensors(), fb.tensors()):
        assert torch.equal(x, y)
    st = ia.stats()
    assert not st["overflow"]


def test_per_view_baseline_runs_the_same_work(gpf):
    """The per-view launch loop updates the same parameters; with one view it
    is the batched step exactly."""
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    from paper_2512_12459_gb300.train import TrainStep, per_view_step
    fnp, qnp, tgt = _scene(seed=44, n_views=1, sides=(48,))
    queries = gpf.Queries.from_numpy(qnp)
    target = _target(gpf, tgt, queries)
    fa, fb = gpf.Field.from_numpy(fnp), gpf.Field.from_numpy(fnp)
    ia = make_index(fa, queries, query_cell=0.05, headroom=1.5)
    ib = make_index(fb, queries, grid=ia.grid)
    step = TrainStep(fa, queries, target, ia, r_max=R, lr=5e-3)
    state = gpf.AdamState.zeros_like(fb, device_counter=True)
    grads = gpf.Field.zeros_like(fb)
    outs = [torch.empty_like(target)]
    zs = [torch.empty((queries.m,), device="cuda")]
    gouts = [torch.empty_like(target)]
    for _ in range(3):
        step()
        per_view_step(fb, [queries], [target], [ib], state, grads, outs, zs, gouts, r_max=R,
                      lr=5e-3)
    torch.cuda.synchronize()
    for x, y in zip(fa.tensors(), fb.tensors()):
        assert torch.equal(x, y)


def test_autotune_chooses_among_candidates_and_keeps_results(gpf):
    from paper_2512_12459_gb300.setup_index import autotune, make_index
    fnp, qnp, _ = _scene(seed=45)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    grid, report = autotune(field, queries, r_max=R, query_cells=(0.02, 0.05),
                            max_spans=(3, 4), coop_options=(2, 4), repeats=1)
    assert len(report) >= 4 and all(ms > 0 for _, ms in report)
    best_ms = min(ms for _, ms in report)
    assert any(ms == best_ms for _, ms in report)
    assert grid.max_span in (3, 4) and grid.coop_cells in (2, 4)
    ia = make_index(field, queries, grid=grid)
    ia.build(field, queries)
    a, _ = gpf.gpf_radiance_fwd(ia, field, queries, gpf.GPF_SUM, r_max=R)
    sel = sample_active(qnp, 300, seed=46)
    ref = oracle_fwd(fnp, qnp, oracle.GPF_SUM, R, 3.0, sel)
    err, zero_ok = fwd_rel_err(a.cpu().numpy().astype(np.float64)[:, sel], ref)
    assert err <= FWD_TOL and zero_ok


@pytest.mark.parametrize("coop", [1, 8])
def test_tile_shape_extremes_match_the_oracle(gpf, coop):
    """coop_cells = 1 (almost every level pooled) and 8 (mostly cooperative)."""
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp, _ = _scene(seed=47)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.03, coop_cells=coop)
    idx.build(field, queries)
    out, _ = gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=R)
    sel = sample_active(qnp, 300, seed=48)
    ref = oracle_fwd(fnp, qnp, oracle.GPF_SUM, R, 3.0, sel)
    err, zero_ok = fwd_rel_err(out.cpu().numpy().astype(np.float64)[:, sel], ref)
    assert err <= FWD_TOL and zero_ok
