"""The data-parallel path on CPU ranks (gloo, world size 2): view sharding,
the count-weighted gradient all-reduce and the timing reductions, checked
against the single-process gradient of the MSE over all views (oracle)."""

import os
import socket

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

from paper_2512_12459_gb300 import sharding  # noqa: E402

WORLD = 2
VIEW_SIZES = [37, 61, 20]   # hit points per view; view 1 has invalid points


def test_shard_views_cover_balance_and_agree():
    sizes = [256 * 256, 1024 * 1024, 384 * 384, 512 * 512, 1024 * 1024, 768 * 768, 256 * 256]
    for world in (1, 2, 3, 4, 8):
        parts = [sharding.shard_views(sizes, world, r) for r in range(world)]
        flat = sorted(v for p in parts for v in p)
        assert flat == list(range(len(sizes)))                 # every view exactly once
        assert parts == [sharding.shard_views(sizes, world, r) for r in range(world)]
        loads = [sum(sizes[v] for v in p) for p in parts]
        # greedy by size: no rank exceeds the average by more than the largest view
        assert max(loads) <= sum(sizes) / world + max(sizes)
    assert sharding.shard_views([5, 5], 2, 0) == [0] and sharding.shard_views([5, 5], 2, 1) == [1]
    with pytest.raises(ValueError):
        sharding.shard_views([1], 2, 2)


def _scene():
    fnp, qnp = synth.config1_random(seed=31, n=40, m=sum(VIEW_SIZES))
    fnp.logscale = (fnp.logscale + 1.5).astype(np.float32)     # wider Gaussians: more pairs
    qnp.valid[[40, 41, 50, 77, 80, 90, 95]] = 0                # invalid points in view 1
    tgt = synth.perturbed_copy(fnp, seed=32)
    bounds = np.cumsum([0] + VIEW_SIZES)
    return fnp, qnp, tgt, bounds


def _grads(fnp, tgt, q):
    """Oracle forward, MSE gradient normalised by q's own valid count, backward."""
    args = dict(mode=oracle.GPF_SUM, r_max=0.3, cutoff_sigma=3.0)
    out = oracle.radiance_fwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, q.x, q.n, q.wo,
                              None, q.valid, **args)["out"]
    ref = oracle.radiance_fwd(tgt.mean, tgt.quat, tgt.logscale, tgt.spectrum, q.x, q.n, q.wo,
                              None, q.valid, **args)["out"]
    g = oracle.mse_loss_grad(out, ref, q.valid)
    gr = oracle.radiance_bwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, q.x, q.n, q.wo, g,
                             None, q.valid, **args)
    return [gr[k] for k in ("mean", "quat", "logscale", "spectrum")]


def _worker(rank, world, port, outdir):
    os.environ.pop("CUDA_VISIBLE_DEVICES", None)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        fnp, qnp, tgt, bounds = _scene()
        mine = sharding.shard_views(VIEW_SIZES, world, rank)
        idx = np.concatenate([np.arange(bounds[v], bounds[v + 1]) for v in mine])
        q = synth.subset_queries(qnp, idx)
        n_local = int(q.valid.sum())
        n_total = sharding.global_count(n_local)
        grads = [torch.as_tensor(a.copy()) for a in _grads(fnp, tgt, q)]
        sharding.allreduce_gradients(grads, n_local, n_total)
        t_max = sharding.max_over_ranks(1.5 + rank)
        q_sum = sharding.sum_over_ranks(float(len(idx)))
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), *[g.numpy() for g in grads],
                 n_total=n_total, t_max=t_max, q_sum=q_sum)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_weighted_allreduce_equals_the_global_mse_gradient(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(WORLD, _free_port(), str(tmp_path)), nprocs=WORLD,
                       join=True, start_method="spawn")
    fnp, qnp, tgt, _ = _scene()
    want = _grads(fnp, tgt, qnp)          # one process, MSE over every view's valid points
    for r in range(WORLD):
        got = np.load(tmp_path / f"rank{r}.npz")
        assert int(got["n_total"]) == int(qnp.valid.sum())
        assert float(got["t_max"]) == 1.5 + WORLD - 1
        assert float(got["q_sum"]) == sum(VIEW_SIZES)
        for i, w in enumerate(want):
            g = got[f"arr_{i}"]
            assert np.abs(w).max() > 0
            np.testing.assert_allclose(g, w, rtol=1e-12, atol=1e-15 * np.abs(w).max())
    # neither the plain sum nor the plain mean of the per-rank gradients is
    # that gradient (the ranks hold different numbers of valid points)
    parts = [sharding.shard_views(VIEW_SIZES, WORLD, r) for r in range(WORLD)]
    _, _, _, bounds = _scene()
    plain = None
    for p in parts:
        idx = np.concatenate([np.arange(bounds[v], bounds[v + 1]) for v in p])
        g = _grads(fnp, tgt, synth.subset_queries(qnp, idx))
        plain = g if plain is None else [a + b for a, b in zip(plain, g)]
    counts = [int(synth.subset_queries(qnp, np.concatenate(
        [np.arange(bounds[v], bounds[v + 1]) for v in p])).valid.sum()) for p in parts]
    assert counts[0] != counts[1]
    assert not np.allclose(plain[3], want[3], rtol=1e-6)
    assert not np.allclose(plain[3] / WORLD, want[3], rtol=1e-6)


def test_single_process_helpers_are_identities():
    g = [torch.ones(3, 4)]
    sharding.allreduce_gradients(g, 5, 5)
    assert torch.equal(g[0], torch.ones(3, 4))
    assert sharding.global_count(7) == 7
    assert sharding.max_over_ranks(2.5) == 2.5 and sharding.sum_over_ranks(3.0) == 3.0
