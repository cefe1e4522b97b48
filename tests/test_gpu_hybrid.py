"""The paper's hybrid neighbourhood (GPF_NB_BALL_KNN: ball(r) or the k_min
nearest means, Sec. 4.2 and Algorithm S3) on the GPU against the oracle,
including the ball-only and kNN-only variants of the paper's ablation."""

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import FWD_TOL, fwd_rel_err, sample_active

pytestmark = pytest.mark.gpu

R = 0.02


@pytest.fixture(scope="module")
def gpf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12459_gb300 as g
    return g


def _run(gpf, fnp, qnp, mode, ball_r, k_min, cell=0.05):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=cell, ball_radius=max(ball_r, 0.02))
    idx.build(field, queries)
    out, z = gpf.gpf_radiance_fwd(idx, field, queries, mode, r_max=R,
                                  neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=ball_r, k_min=k_min)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), (idx, field, queries, out, z)


def _check(fnp, qnp, out, mode, ball_r, k_min, sel):
    ref = oracle.hybrid_fwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, qnp.x[:, sel],
                            qnp.n[:, sel], qnp.wo[:, sel], None, qnp.valid[sel], mode=mode,
                            r_max=R, ball_r=ball_r, k_min=k_min)
    keep = ~ref["near"]
    err, zero_ok = fwd_rel_err(out[:, sel], {**ref, "near_cutoff": ref["near"]}, keep)
    assert keep.mean() > 0.9
    assert err <= FWD_TOL and zero_ok
    return ref


@pytest.mark.parametrize("mode", [oracle.GPF_NORMALIZED, oracle.GPF_SUM])
def test_hybrid_on_a_caustic_field(gpf, mode):
    pos, flux = synth.caustic_photons(20000, seed=91)
    fnp = synth.field_from_photons(pos, flux, seed=91)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 112, 96)
    out, _ = _run(gpf, fnp, qnp, mode, R, 3)
    sel = sample_active(qnp, 400, seed=92)
    ref = _check(fnp, qnp, out, mode, R, 3, sel)
    # both regimes occur: dense balls and kNN fallback
    assert ref["knn"].any() and (~ref["knn"] & (ref["n_nb"] > 3)).any()


@pytest.mark.parametrize("ball_r,k_min", [(R, 0), (0.0, 3), (R, 8)])
def test_ablation_variants(gpf, ball_r, k_min):
    """ball only (w_radius), kNN only (w_knn), and a larger k_min."""
    pos, flux = synth.caustic_photons(8000, seed=93)
    fnp = synth.field_from_photons(pos, flux, seed=93)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 80, 64)
    out, _ = _run(gpf, fnp, qnp, oracle.GPF_NORMALIZED, ball_r, k_min)
    sel = sample_active(qnp, 300, seed=94)
    _check(fnp, qnp, out, oracle.GPF_NORMALIZED, ball_r, k_min, sel)


def test_sparse_field_falls_back_to_knn(gpf):
    fnp, qnp = synth.config1_random(seed=95, n=300, m=2000)
    out, _ = _run(gpf, fnp, qnp, oracle.GPF_NORMALIZED, R, 3, cell=0.1)
    sel = sample_active(qnp, 300, seed=96)
    ref = _check(fnp, qnp, out, oracle.GPF_NORMALIZED, R, 3, sel)
    assert ref["knn"].mean() > 0.9


@pytest.mark.parametrize("mode", [oracle.GPF_NORMALIZED, oracle.GPF_SUM])
def test_dense_tiles_are_split_and_match_the_oracle(gpf, mode):
    """A dense caustic (30,000 photons with a 3 cm spread) seen from close
    by: every tile's ball box lists thousands of means, so the forward splits
    the tiles into parts over their entries and adds the parts' sums in
    order; each hit point still sums its whole ball (or its k_min nearest at
    the rim)."""
    pos, flux = _dense_blob(30000, 97)
    fnp = synth.field_from_photons(pos, flux, seed=97)
    qnp = synth.pinhole_hitpoints((2.0, -0.15, 0.15), (2.0, 0.0, 0.0), 64, 48)
    out, (idx, *_rest) = _run(gpf, fnp, qnp, mode, R, 3)
    assert idx.stats()["n_hybrid_units"] > 0
    sel = sample_active(qnp, 300, seed=98)
    _check(fnp, qnp, out, mode, R, 3, sel)


def test_hybrid_backward_needs_pair_room_and_centre_entries(gpf):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp = synth.config1_random(seed=97, n=200, m=500)
    out, (idx, field, queries, o, z) = _run(gpf, fnp, qnp, oracle.GPF_SUM, R, 3, cell=0.1)
    with pytest.raises(gpf.GPFError):
        gpf.gpf_radiance_bwd(idx, field, queries, torch.ones_like(o), o, z, gpf.GPF_SUM, r_max=R,
                             neighbourhood=gpf.GPF_NB_BALL_KNN)
    plain = make_index(field, queries, query_cell=0.1)
    plain.build(field, queries)
    with pytest.raises(gpf.GPFError):
        gpf.gpf_radiance_fwd(plain, field, queries, gpf.GPF_SUM, r_max=R,
                             neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=R, k_min=3)
    with pytest.raises(gpf.GPFError):     # a ball wider than the index's
        gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=R,
                             neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=0.5, k_min=3)


def test_hybrid_with_no_gaussians_returns_zeros(gpf):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp = synth.config1_random(seed=98, n=0, m=300)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.1, ball_radius=R)
    idx.build(field, queries)
    out, z = gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_NORMALIZED, r_max=R,
                                  neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=R, k_min=3)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0 and torch.count_nonzero(z).item() == 0


def _bwd_case(gpf, fnp, qnp, mode, ball_r, k_min, cell=0.05, seed=0, f64=False, room=4.0):
    """GPU gradients of the hybrid query and the oracle's, with the upstream
    gradient zeroed at hit points whose selection float32 may decide
    differently (a mean at the ball's edge, a k-th / (k+1)-th distance tie)."""
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    ref_f = oracle.hybrid_fwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, qnp.x, qnp.n,
                              qnp.wo, None, qnp.valid, mode=mode, r_max=R, ball_r=ball_r,
                              k_min=k_min)
    G = np.random.default_rng(seed).standard_normal((fnp.channels, qnp.m))
    G[:, ref_f["near"]] = 0.0
    G = G.astype(np.float32)
    cap = int(room * max(1, ref_f["n_nb"].sum())) + 1024
    idx = make_index(field, queries, query_cell=cell, ball_radius=max(ball_r, 0.02),
                     max_nb_pairs=cap)
    idx.build(field, queries)
    out, z = gpf.gpf_radiance_fwd(idx, field, queries, mode, r_max=R,
                                  neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=ball_r, k_min=k_min)
    if f64:
        # the gradient-check build is given the oracle's forward (rounded to
        # float32), so that it checks the backward alone
        out = torch.as_tensor(ref_f["out"], dtype=torch.float32, device="cuda").contiguous()
        z = torch.as_tensor(ref_f["Z"], dtype=torch.float32, device="cuda").contiguous()
    g = gpf.gpf_radiance_bwd(idx, field, queries, torch.as_tensor(G, device="cuda"), out, z, mode,
                             r_max=R, neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=ball_r,
                             k_min=k_min, f64_sums=f64)
    torch.cuda.synchronize()
    ref = oracle.hybrid_bwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, qnp.x, qnp.n,
                            qnp.wo, G, None, qnp.valid, mode=mode, r_max=R, ball_r=ball_r,
                            k_min=k_min)
    gg = {k: getattr(g, k).cpu().numpy().astype(np.float64)
          for k in ("mean", "quat", "logscale", "spectrum")}
    return gg, ref, ref_f, idx


def _anisotropic(fnp, seed):
    rng = np.random.default_rng(seed)
    fnp.logscale = (fnp.logscale + rng.normal(0.0, 0.3, fnp.logscale.shape)).astype(np.float32)
    return fnp


@pytest.mark.parametrize("mode", [oracle.GPF_NORMALIZED, oracle.GPF_SUM])
@pytest.mark.parametrize("ball_r,k_min", [(R, 3), (R, 0), (0.0, 3)])
def test_hybrid_backward_matches_the_oracle(gpf, mode, ball_r, k_min):
    """Sec. 4.2, Differentiable Accumulation over N(x) = ball(r) or kNN(k_min)
    held fixed, and the ablation's ball-only and kNN-only selections."""
    from gpu_helpers import GRAD_TOL, grad_err
    pos, flux = synth.caustic_photons(4000, seed=191)
    fnp = _anisotropic(synth.field_from_photons(pos, flux, seed=191), 191)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 64, 48)
    g, ref, ref_f, idx = _bwd_case(gpf, fnp, qnp, mode, ball_r, k_min)
    if k_min and ball_r:
        assert ref_f["knn"].any() and (~ref_f["knn"] & (ref_f["n_nb"] > k_min)).any()
    for k in g:
        assert grad_err(g[k], ref[k]) < GRAD_TOL, (k, grad_err(g[k], ref[k]))


def _dense_blob(n, seed):
    """n photons with a 3 cm spread on the floor at (2, 0), clear of the sphere."""
    rng = np.random.default_rng(seed)
    pos = np.zeros((n, 3))
    pos[:, :2] = rng.standard_normal((n, 2)) * 0.03
    pos[:, 0] += 2.0
    return pos, rng.exponential(1.0, (n, 3))


@pytest.mark.parametrize("mode", [oracle.GPF_NORMALIZED, oracle.GPF_SUM])
def test_dense_tiles_backward_matches_the_oracle(gpf, mode):
    """The backward's selection passes split the dense tiles like the forward:
    each part counts, then writes, the ball pairs of its share of the tile's
    entries after those of the earlier parts. Same pairs, same gradients."""
    from gpu_helpers import GRAD_TOL, grad_err
    pos, flux = _dense_blob(12000, 195)
    fnp = _anisotropic(synth.field_from_photons(pos, flux, seed=195), 195)
    qnp = synth.pinhole_hitpoints((2.0, -0.15, 0.15), (2.0, 0.0, 0.0), 48, 36)
    g, ref, ref_f, idx = _bwd_case(gpf, fnp, qnp, mode, R, 3, seed=5)
    st = idx.stats()
    assert st["n_hybrid_units"] > 0
    assert ref_f["knn"].any() and (ref_f["n_nb"] > 500).any()
    # every point's selection but those float32 may decide differently
    assert abs(st["n_nb_pairs"] - int(ref_f["n_nb"].sum())) <= 16 * int(ref_f["near"].sum())
    for k in g:
        assert grad_err(g[k], ref[k]) < GRAD_TOL, (k, grad_err(g[k], ref[k]))


@pytest.mark.parametrize("mode", [oracle.GPF_NORMALIZED, oracle.GPF_SUM])
def test_hybrid_backward_float64_sums(gpf, mode):
    """The gradient-check build on the hybrid pairs: 1e-6 normwise."""
    from gpu_helpers import grad_err
    pos, flux = synth.caustic_photons(4000, seed=192)
    fnp = _anisotropic(synth.field_from_photons(pos, flux, seed=192), 192)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 64, 48)
    g, ref, _, _ = _bwd_case(gpf, fnp, qnp, mode, R, 3, f64=True, seed=3)
    for k in g:
        assert grad_err(g[k], ref[k]) < 1e-6, (k, grad_err(g[k], ref[k]))


def test_hybrid_backward_is_reproducible_and_flags_a_full_pair_buffer(gpf):
    import torch
    from paper_2512_12459_gb300 import _abi
    from paper_2512_12459_gb300.setup_index import make_index
    pos, flux = synth.caustic_photons(5000, seed=193)
    fnp = synth.field_from_photons(pos, flux, seed=193)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 64, 64)
    g1, _, _, _ = _bwd_case(gpf, fnp, qnp, oracle.GPF_NORMALIZED, R, 3, seed=4)
    g2, _, _, _ = _bwd_case(gpf, fnp, qnp, oracle.GPF_NORMALIZED, R, 3, seed=4)
    for k in g1:
        assert np.array_equal(g1[k], g2[k])
    # room for fewer pairs than the neighbourhoods hold: flagged, untouched
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.05, ball_radius=R, max_nb_pairs=100)
    idx.build(field, queries)
    out, z = gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=R,
                                  neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=R, k_min=3)
    grads = gpf.Field(*(torch.full_like(t, 7.0) for t in field.tensors()))
    gpf.gpf_radiance_bwd(idx, field, queries, torch.ones_like(out), out, z, gpf.GPF_SUM, r_max=R,
                         neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=R, k_min=3, grads=grads)
    torch.cuda.synchronize()
    assert all(torch.all(t == 7.0) for t in grads.tensors())
    assert idx.stats()["flags"] & _abi.GPF_FLAG_CAPACITY


def test_backward_reuses_the_forwards_counts_only_for_the_same_selection(gpf):
    """After a GPF_NB_BALL_KNN forward with the same ball_r and k_min the
    backward takes that forward's per-point counts instead of counting again;
    after a forward with another k_min, or with no forward since the build,
    it counts itself. The gradients are bitwise the same in all three."""
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    pos, flux = _dense_blob(6000, 196)
    fnp = synth.field_from_photons(pos, flux, seed=196)
    qnp = synth.pinhole_hitpoints((2.0, -0.15, 0.15), (2.0, 0.0, 0.0), 48, 36)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.05, ball_radius=R, max_nb_pairs=4_000_000)
    G = torch.as_tensor(np.random.default_rng(7).standard_normal((3, queries.m)),
                        dtype=torch.float32, device="cuda")
    kw = dict(neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=R, k_min=3)

    def grads(forward_k):
        idx.build(field, queries)
        if forward_k is not None:
            gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=R,
                                 neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=R, k_min=forward_k)
        g = gpf.gpf_radiance_bwd(idx, field, queries, G, mode=gpf.GPF_SUM, r_max=R, **kw)
        torch.cuda.synchronize()
        assert idx.stats()["flags"] == 0
        return [t.clone() for t in g.tensors()], idx.stats()["n_nb_pairs"]

    same, n_same = grads(3)
    other, n_other = grads(8)
    none, n_none = grads(None)
    assert n_same == n_other == n_none > 0
    for a, b, c in zip(same, other, none):
        assert torch.equal(a, b) and torch.equal(a, c)
