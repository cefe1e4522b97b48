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


def test_hybrid_has_no_backward_and_needs_centre_entries(gpf):
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
