"""The training run at full size (the measurement plan's third
configuration): 1,000,000 Gaussians fitted over 8 orbit views of 800 x 800
for 200 Adam steps through the captured training step. The loss falls, no
pair buffer overflows, and the forward of the trained field equals the
oracle on sampled hit points of every view."""

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import FWD_TOL, fwd_rel_err, oracle_fwd

pytestmark = pytest.mark.gpu

R = 0.02


@pytest.fixture(scope="module")
def gpf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12459_gb300 as g
    return g


def test_eight_view_training_run_full_size(gpf):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    from paper_2512_12459_gb300.train import TrainStep
    pos, flux = synth.caustic_photons(1_000_000, seed=0)
    fnp = synth.field_from_photons(pos, flux, seed=0)
    tgt_np = synth.perturbed_copy(fnp, seed=1)
    qnp = synth.orbit_views(8, 800, 800)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    tf = gpf.Field.from_numpy(tgt_np)
    tidx = make_index(tf, queries, query_cell=0.02)
    tidx.build(tf, queries)
    target = gpf.gpf_radiance_fwd(tidx, tf, queries, gpf.GPF_SUM, r_max=R)[0].clone()
    del tidx, tf
    idx = make_index(field, queries, query_cell=0.03, max_span=3, coop_cells=8, headroom=1.25)
    step = TrainStep(field, queries, target, idx, r_max=R, lr=5e-4)
    step.capture(warmup=1)
    losses = torch.empty((200,), dtype=torch.float32, device="cuda")
    for i in range(200):
        step()
        losses[i].copy_(step.loss[0])
    torch.cuda.synchronize()
    lh = losses.cpu().numpy()
    assert not idx.stats()["overflow"]
    assert np.all(np.isfinite(lh))
    assert lh[-1] < 0.9 * lh[0], (lh[0], lh[-1])
    assert step.updates() == 201

    # the trained parameters, through a fresh index, against the oracle
    trained = synth.Field(*(t.cpu().numpy() for t in field.tensors()))
    fidx = make_index(field, queries, query_cell=0.03, max_span=3, coop_cells=8)
    fidx.build(field, queries)
    out, _ = gpf.gpf_radiance_fwd(fidx, field, queries, gpf.GPF_SUM, r_max=R)
    out = out.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(7)
    offs = qnp.view_offsets
    sel = []
    for v in range(len(offs) - 1):               # 6 valid points of every view
        act = np.flatnonzero(qnp.valid[offs[v]:offs[v + 1]]) + offs[v]
        sel.extend(rng.choice(act, size=6, replace=False).tolist())
    sel = np.asarray(sorted(sel))
    ref = oracle_fwd(trained, qnp, oracle.GPF_SUM, R, 3.0, sel)
    err, zero_ok = fwd_rel_err(out[:, sel], ref)
    assert err <= FWD_TOL and zero_ok, err
