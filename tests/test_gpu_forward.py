"""Forward parity of the CUDA path (through the C ABI) against the FP64 oracle."""

import math

import numpy as np
import pytest

import oracle
import synth
from golden_util import load_examples
from gpu_helpers import (FWD_TOL, GRAD_TOL, INF, fwd_rel_err, gpu_fwd, oracle_fwd,
                         sample_active)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12459_gb300 as g
    return g


def test_worked_examples_on_gpu(gpf):
    examples, _ = load_examples()
    for name, ex in examples.items():
        f = synth.Field(ex["mean"], ex["quat"], ex["logscale"], ex["spectrum"])
        q = synth.Queries(ex["x"], ex["n"], ex["wo"], ex["albedo"],
                          np.ones(ex["x"].shape[1], np.uint8))
        for brute in (True, False):
            if not brute and math.isinf(ex["cutoff_sigma"]):
                continue
            out, _, _, _ = gpu_fwd(gpf, f, q, ex["mode"], ex["r_max"], ex["cutoff_sigma"],
                                   cell=0.05, brute=brute)
            np.testing.assert_allclose(out, ex["expected"], rtol=FWD_TOL, atol=1e-30,
                                       err_msg=f"{name} brute={brute}")


@pytest.mark.parametrize("mode", [oracle.GPF_SUM, oracle.GPF_NORMALIZED])
@pytest.mark.parametrize("r_max", [INF, 0.02])
def test_config1_brute_force(gpf, mode, r_max):
    """4,096 Gaussians, 16,384 (+13 ragged) hit points, no truncation."""
    fnp, qnp = synth.config1_random(seed=0, n=4096, m=16384 + 13, albedo=True)
    out, z, _, _ = gpu_fwd(gpf, fnp, qnp, mode, r_max, INF)
    sel = sample_active(qnp, 2500, seed=1)
    ref = oracle_fwd(fnp, qnp, mode, r_max, INF, sel)
    err, zero_ok = fwd_rel_err(out[:, sel], ref)
    assert err < FWD_TOL and zero_ok, err
    act = ref["mask"]
    np.testing.assert_allclose(z[sel][act], ref["Z"][act], rtol=FWD_TOL, atol=1e-30)
    # inactive points (back-facing: about half of them) are exactly zero
    ref_all_mask = (np.sum(qnp.n.astype(np.float64) * qnp.wo, axis=0) > 0)
    assert np.all(out[:, ~ref_all_mask] == 0.0)


@pytest.mark.parametrize("cell", [0.03, 0.1, 0.35])
@pytest.mark.parametrize("mode", [oracle.GPF_SUM, oracle.GPF_NORMALIZED])
def test_config1_culled(gpf, cell, mode):
    fnp, qnp = synth.config1_random(seed=2, n=4096, m=8192 + 5, albedo=True)
    out, _, idx, _ = gpu_fwd(gpf, fnp, qnp, mode, 0.02, 3.0, cell=cell)
    sel = sample_active(qnp, 2000, seed=3)
    ref = oracle_fwd(fnp, qnp, mode, 0.02, 3.0, sel)
    err, zero_ok = fwd_rel_err(out[:, sel], ref)
    assert err < FWD_TOL and zero_ok, (err, idx.stats())
    assert ref["near_cutoff"].sum() < 0.01 * sel.size


def test_culled_equals_brute_force_on_gpu(gpf):
    """Grid-culled sum = brute-force sum with the same Q <= 9 predicate, for
    several cell sizes (same pairs; only the summation order differs)."""
    fnp, qnp = synth.config1_random(seed=4, n=3000, m=6000)
    ob, zb, _, _ = gpu_fwd(gpf, fnp, qnp, oracle.GPF_SUM, 0.05, 3.0, brute=True)
    for cell in (0.02, 0.07, 0.2, 0.6):
        oc, zc, _, _ = gpu_fwd(gpf, fnp, qnp, oracle.GPF_SUM, 0.05, 3.0, cell=cell)
        np.testing.assert_allclose(oc, ob, rtol=2e-6, atol=1e-30, err_msg=f"cell {cell}")
        np.testing.assert_allclose(zc, zb, rtol=2e-6, atol=1e-30)


def _caustic(n_photons, seed, w, h, channels=3, merge=False):
    pos, flux = synth.caustic_photons(n_photons, seed=seed, channels=channels)
    if merge:
        pos, flux = synth.merge_photon_pairs(pos, flux)
    f = synth.field_from_photons(pos, flux, seed=seed)
    q = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), w, h)
    return f, q


@pytest.mark.parametrize("mode", [oracle.GPF_SUM, oracle.GPF_NORMALIZED])
def test_caustic_scene_sampled(gpf, mode):
    fnp, qnp = _caustic(40000, seed=5, w=192, h=160)
    out, _, idx, _ = gpu_fwd(gpf, fnp, qnp, mode, 0.02, 3.0, cell=0.05)
    sel = sample_active(qnp, 500, seed=6)
    ref = oracle_fwd(fnp, qnp, mode, 0.02, 3.0, sel)
    err, zero_ok = fwd_rel_err(out[:, sel], ref)
    assert err < FWD_TOL and zero_ok, (err, idx.stats())
    assert np.mean(ref["n_pairs"][ref["mask"]]) > 5


def test_full_size_caustic_scene_sampled(gpf):
    """1,000,000 Gaussians, 1024 x 1024 view (the benchmark workload), grid-culled
    at 3 sigma, r = 0.02; 40 sampled hit points against the oracle."""
    fnp, qnp = _caustic(1000000, seed=0, w=1024, h=1024)
    out, _, idx, _ = gpu_fwd(gpf, fnp, qnp, oracle.GPF_SUM, 0.02, 3.0, cell=0.04)
    st = idx.stats()
    assert not st["overflow"]
    sel = sample_active(qnp, 40, seed=7, tail=4)
    ref = oracle_fwd(fnp, qnp, oracle.GPF_SUM, 0.02, 3.0, sel)
    err, zero_ok = fwd_rel_err(out[:, sel], ref)
    assert err < FWD_TOL and zero_ok, err


def test_merged_field_and_eight_channels(gpf):
    fnp, qnp = _caustic(20000, seed=8, w=96, h=96, channels=8, merge=True)
    assert fnp.n == 10000 and fnp.channels == 8
    out, _, _, _ = gpu_fwd(gpf, fnp, qnp, oracle.GPF_NORMALIZED, 0.02, 3.0, cell=0.05)
    sel = sample_active(qnp, 400, seed=9)
    ref = oracle_fwd(fnp, qnp, oracle.GPF_NORMALIZED, 0.02, 3.0, sel)
    err, zero_ok = fwd_rel_err(out[:, sel], ref)
    assert err < FWD_TOL and zero_ok, err


@pytest.mark.parametrize("channels", [1, 2, 5, 7])
def test_channel_counts(gpf, channels):
    fnp, qnp = synth.config1_random(seed=10 + channels, n=700, m=1500, channels=channels,
                                    albedo=True)
    for brute in (True, False):
        out, _, _, _ = gpu_fwd(gpf, fnp, qnp, oracle.GPF_SUM, 0.05, 3.0, cell=0.1, brute=brute)
        ref = oracle_fwd(fnp, qnp, oracle.GPF_SUM, 0.05, 3.0)
        err, zero_ok = fwd_rel_err(out, ref)
        assert err < FWD_TOL and zero_ok, (channels, brute, err)


def test_points_outside_the_grid_are_clamped_exactly(gpf):
    """A grid covering only the middle of the scene: border cells absorb the
    rest and the result is unchanged."""
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp = synth.config1_random(seed=20, n=2000, m=4000)
    field = gpf.Field.from_numpy(fnp)
    queries = gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.05, cutoff_sigma=3.0,
                     bounds=([0.3, 0.3, 0.3], [0.7, 0.7, 0.7]))
    idx.build(field, queries)
    out, _ = gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=0.05)
    ref = oracle_fwd(fnp, qnp, oracle.GPF_SUM, 0.05, 3.0)
    err, zero_ok = fwd_rel_err(out.cpu().numpy().astype(np.float64), ref)
    assert err < FWD_TOL and zero_ok


def test_empty_and_degenerate_inputs(gpf):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp = synth.config1_random(seed=21, n=100, m=300)
    # no Gaussians: zero radiance
    f0 = synth.Field(*(a[:, :0].copy() for a in (fnp.mean, fnp.quat, fnp.logscale,
                                                 fnp.spectrum)))
    out, z, _, _ = gpu_fwd(gpf, f0, qnp, oracle.GPF_NORMALIZED, INF, 3.0, cell=0.1)
    assert np.all(out == 0) and np.all(z == 0)
    # no hit points
    q0 = synth.subset_queries(qnp, np.arange(0))
    field = gpf.Field.from_numpy(fnp)
    queries = gpf.Queries.from_numpy(q0)
    idx = make_index(field, queries, query_cell=0.1, bounds=([0, 0, 0], [1, 1, 1]))
    idx.build(field, queries)
    o, zz = gpf.gpf_radiance_fwd(idx, field, queries)
    assert o.shape == (3, 0)
    # every hit point invalid
    qi = synth.subset_queries(qnp, np.arange(qnp.m))
    qi.valid = np.zeros(qnp.m, np.uint8)
    out, z, idx, _ = gpu_fwd(gpf, fnp, qi, oracle.GPF_SUM, INF, 3.0, cell=0.1)
    assert np.all(out == 0) and idx.stats()["n_active"] == 0
    # one Gaussian, one hit point on top of it
    f1 = synth.subset_field(fnp, np.array([5]))
    q1 = synth.Queries(fnp.mean[:, [5]].copy(), np.array([[0], [0], [1]], np.float32),
                       np.array([[0], [0], [1]], np.float32), None, np.ones(1, np.uint8))
    out, z, _, _ = gpu_fwd(gpf, f1, q1, oracle.GPF_SUM, INF, 3.0, cell=0.1)
    np.testing.assert_allclose(out[:, 0], f1.spectrum[:, 0], rtol=1e-6)
    del torch


def test_forward_is_bitwise_reproducible(gpf):
    fnp, qnp = _caustic(30000, seed=22, w=128, h=128)
    a, za, _, _ = gpu_fwd(gpf, fnp, qnp, oracle.GPF_NORMALIZED, 0.02, 3.0, cell=0.05)
    b, zb, _, _ = gpu_fwd(gpf, fnp, qnp, oracle.GPF_NORMALIZED, 0.02, 3.0, cell=0.05)
    assert np.array_equal(a, b) and np.array_equal(za, zb)


def test_timing_events_bracket_the_pair_loops(gpf):
    """gpf_index_set_timing_events: the events are recorded around the pair
    loops of both calls and measure a positive time; clearing them stops it."""
    import torch
    fnp, qnp = _caustic(30000, seed=23, w=128, h=128)
    out, z, idx, (field, queries, out_t, z_t) = gpu_fwd(gpf, fnp, qnp, oracle.GPF_SUM, 0.02, 3.0,
                                                         cell=0.05)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    idx.set_timing_events(fwd=(ev[0], ev[1]), bwd=(ev[2], ev[3]))
    gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=0.02, out=out_t, z=z_t)
    gpf.gpf_radiance_bwd(idx, field, queries, torch.ones_like(out_t), out_t, z_t, gpf.GPF_SUM,
                         r_max=0.02)
    torch.cuda.synchronize()
    assert ev[0].elapsed_time(ev[1]) > 0 and ev[2].elapsed_time(ev[3]) > 0
    idx.set_timing_events()
    gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=0.02, out=out_t, z=z_t)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out_t.cpu().numpy(), out.astype(np.float32))


def test_overflow_is_reported_and_outputs_untouched(gpf):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp = synth.config1_random(seed=23, n=2000, m=3000)
    field = gpf.Field.from_numpy(fnp)
    queries = gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.03, cutoff_sigma=3.0, max_pairs=64)
    idx.build(field, queries)
    st = idx.stats()
    assert st["overflow"] and st["n_pairs"] > 64
    out = torch.full((3, qnp.m), float("nan"), device="cuda")
    gpf.gpf_radiance_fwd(idx, field, queries, out=out)
    torch.cuda.synchronize()
    assert torch.isnan(out).all()


def test_mismatched_inputs_are_refused(gpf):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp = synth.config1_random(seed=24, n=200, m=300)
    field = gpf.Field.from_numpy(fnp)
    queries = gpf.Queries.from_numpy(qnp)
    other = gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.1)
    with pytest.raises(gpf.GPFError, match="NOT_BUILT"):
        gpf.gpf_radiance_fwd(idx, field, queries)
    idx.build(field, queries)
    with pytest.raises(gpf.GPFError, match="MISMATCH"):
        gpf.gpf_radiance_fwd(idx, field, other)
    with pytest.raises(gpf.GPFError, match="INVALID_ARG"):
        gpf.gpf_radiance_fwd(idx, field, queries, mode=7)
    torch.cuda.synchronize()


@pytest.mark.parametrize("mode", [oracle.GPF_SUM, oracle.GPF_NORMALIZED])
def test_split_tiles_equal_unsplit_and_the_oracle(gpf, mode):
    """Forward load balancing: tiles whose estimated work exceeds split_items
    run as up to GPF_MAX_TILE_PARTS units over disjoint chunks of their
    lists, summed in part order. Same pairs as the unsplit forward (pair
    counts equal), sums equal up to their order, parity with the oracle, and
    bitwise reproducible."""
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp = _caustic(40000, seed=15, w=160, h=128)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    outs = {}
    for split in (0, 64, 512):
        idx = make_index(field, queries, query_cell=0.05, split_items=split)
        idx.build(field, queries)
        o, z = gpf.gpf_radiance_fwd(idx, field, queries, mode, r_max=0.02)
        o2, _ = gpf.gpf_radiance_fwd(idx, field, queries, mode, r_max=0.02)
        torch.cuda.synchronize()
        assert torch.equal(o, o2)
        outs[split] = (o.cpu().numpy().astype(np.float64), z.cpu().numpy().astype(np.float64),
                       gpf.gpf_count_pairs(idx, field, queries))
    base_o, base_z, base_c = outs[0]
    for split in (64, 512):
        o, z, c = outs[split]
        assert c == base_c
        np.testing.assert_allclose(o, base_o, rtol=2e-6, atol=1e-30)
        np.testing.assert_allclose(z, base_z, rtol=2e-6, atol=1e-30)
    sel = sample_active(qnp, 400, seed=16)
    ref = oracle_fwd(fnp, qnp, mode, 0.02, 3.0, sel)
    err, zero_ok = fwd_rel_err(outs[64][0][:, sel], ref)
    assert err < FWD_TOL and zero_ok, err


def test_tile_order_changes_summation_order_only(gpf):
    """Hit points ordered inside their query cells by 2^b sub-cells (b = 1, 2)
    instead of by index: the same pairs (included pair counts equal; the
    candidates the tile boxes let through differ), outputs and
    gradients equal to the index order's up to summation order, and parity
    with the oracle."""
    import dataclasses

    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp = _caustic(40000, seed=21, w=160, h=128)
    # anisotropic scales, so that the rotation gradient is not rounding noise
    rng = np.random.default_rng(21)
    fnp.logscale = (fnp.logscale + rng.normal(0.0, 0.3, fnp.logscale.shape)).astype(np.float32)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    base = make_index(field, queries, query_cell=0.05, split_items=256)
    orders = [b for b in (0, 1, 2) if b <= base.grid.query_level]
    assert len(orders) >= 2
    gout = torch.as_tensor(rng.standard_normal((3, queries.m)).astype(np.float32), device="cuda")
    res = {}
    for b in orders:
        idx = make_index(field, queries, grid=dataclasses.replace(base.grid, tile_order=b))
        idx.build(field, queries)
        o, z = gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=0.02)
        g = gpf.gpf_radiance_bwd(idx, field, queries, gout, o, z, gpf.GPF_SUM, r_max=0.02)
        torch.cuda.synchronize()
        res[b] = (o.cpu().numpy().astype(np.float64), gpf.gpf_count_pairs(idx, field, queries),
                  [t.cpu().numpy().astype(np.float64) for t in g.tensors()])
    o0, c0, g0 = res[0]
    for b in orders[1:]:
        o, c, g = res[b]
        assert c["included"] == c0["included"]
        np.testing.assert_allclose(o, o0, rtol=2e-6, atol=1e-30)
        for t, t0 in zip(g, g0):
            assert np.linalg.norm(t - t0) <= GRAD_TOL * np.linalg.norm(t0)
    sel = sample_active(qnp, 400, seed=22)
    ref = oracle_fwd(fnp, qnp, oracle.GPF_SUM, 0.02, 3.0, sel)
    err, zero_ok = fwd_rel_err(res[orders[-1]][0][:, sel], ref)
    assert err < FWD_TOL and zero_ok, err
