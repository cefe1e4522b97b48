"""16-bit parameter storage (GPF_BF16): the GPU quantiser against the host
encoder, the decoded path against the float32 path and the oracle, the
quantisation error against the oracle on the float32 parameters, and the
training step with a bfloat16 copy."""

import numpy as np
import pytest

import oracle
import synth
from synth import storage
from gpu_helpers import FWD_TOL, GRAD_TOL, fwd_rel_err, grad_err, oracle_fwd, sample_active

pytestmark = pytest.mark.gpu

R = 0.02


@pytest.fixture(scope="module")
def gpf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12459_gb300 as g
    return g


def _field(n_photons, seed, channels=3, aniso=0.0):
    pos, flux = synth.caustic_photons(n_photons, seed=seed, channels=channels)
    f = synth.field_from_photons(pos, flux, seed=seed)
    if aniso:
        rng = np.random.default_rng(seed + 1000)
        f.logscale = (f.logscale + rng.normal(0.0, aniso, f.logscale.shape)).astype(np.float32)
    return storage.permuted(f, storage.morton_order(f))


def _upload_bf16(gpf, b):
    import torch
    t = lambda a: torch.from_numpy(a.view(np.int16).copy()).view(torch.bfloat16).cuda()  # noqa
    mean = torch.from_numpy(b.mean).cuda() if b.mean.dtype == np.float32 else t(b.mean)
    return gpf.Field(mean, t(b.quat), t(b.logscale), t(b.spectrum),
                     torch.from_numpy(b.anchor.copy()).cuda())


@pytest.mark.parametrize("mean32", [False, True])
def test_gpu_quantiser_equals_host_encoder(gpf, mean32):
    import torch
    f = _field(5003, seed=61, aniso=0.3)             # a ragged last group
    f.quat = (f.quat * 3.7).astype(np.float32)        # non-unit quaternions are stored as given
    want = storage.encode(f, mean32=mean32)
    got = gpf.Field.from_numpy(f).quantized(mean32=mean32)
    assert got.storage == (2 if mean32 else 1)
    torch.cuda.synchronize()
    for name in ("mean", "quat", "logscale", "spectrum"):
        t = getattr(got, name)
        a = t.cpu().numpy() if t.dtype == torch.float32 else \
            t.view(torch.int16).cpu().numpy().view(np.uint16)
        assert a.dtype == getattr(want, name).dtype and np.array_equal(a, getattr(want, name)), name
    assert np.array_equal(got.anchor.cpu().numpy(), want.anchor)
    dec = got.decoded()
    ref = storage.decode(want)
    for name in ("mean", "quat", "logscale", "spectrum"):
        assert np.array_equal(getattr(dec, name).cpu().numpy(), getattr(ref, name)), name


@pytest.mark.parametrize("mode,mean32", [(oracle.GPF_SUM, False), (oracle.GPF_NORMALIZED, False),
                                         (oracle.GPF_SUM, True)])
def test_bf16_path_equals_float32_path_on_decoded_values(gpf, mode, mean32):
    """The 16-bit field is decoded once at build: forward and backward then
    equal the float32 path run on the decoded parameters bit for bit, and the
    oracle on those parameters within the forward tolerance."""
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    f = _field(30000, seed=62, aniso=0.3)
    b = storage.encode(f, mean32=mean32)
    dnp = storage.decode(b)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 160, 128)
    queries = gpf.Queries.from_numpy(qnp)
    fb = _upload_bf16(gpf, b)
    fd = gpf.Field.from_numpy(dnp)
    ib = make_index(fb, queries, query_cell=0.05)
    idd = make_index(fd, queries, grid=ib.grid)
    assert ib.grid.field_storage == (2 if mean32 else 1) and idd.grid.field_storage == 0
    outs = []
    for fld, idx in ((fb, ib), (fd, idd)):
        idx.build(fld, queries)
        o, z = gpf.gpf_radiance_fwd(idx, fld, queries, mode, r_max=R)
        g = gpf.gpf_radiance_bwd(idx, fld, queries, torch.ones_like(o), o, z, mode, r_max=R)
        outs.append((o, z, g))
    torch.cuda.synchronize()
    (ob, zb, gb), (od, zd, gd) = outs
    assert torch.equal(ob, od) and torch.equal(zb, zd)
    for x, y in zip(gb.tensors(), gd.tensors()):
        assert x.dtype == torch.float32 and torch.equal(x, y)
    sel = sample_active(qnp, 300, seed=63)
    ref = oracle_fwd(dnp, qnp, mode, R, 3.0, sel)
    err, zero_ok = fwd_rel_err(ob.cpu().numpy().astype(np.float64)[:, sel], ref)
    assert err <= FWD_TOL and zero_ok


def test_bf16_gradients_match_the_oracle_on_decoded_values(gpf):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    f = _field(3000, seed=64, aniso=0.3)
    b = storage.encode(f)
    dnp = storage.decode(b)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 48, 40)
    queries = gpf.Queries.from_numpy(qnp)
    fb = _upload_bf16(gpf, b)
    idx = make_index(fb, queries, query_cell=0.1)
    idx.build(fb, queries)
    o, z = gpf.gpf_radiance_fwd(idx, fb, queries, gpf.GPF_SUM, r_max=R)
    rng = np.random.default_rng(65)
    gout = rng.standard_normal(tuple(o.shape)).astype(np.float32)
    g = gpf.gpf_radiance_bwd(idx, fb, queries, torch.as_tensor(gout, device="cuda"), o, z,
                             gpf.GPF_SUM, r_max=R)
    ref = oracle.radiance_bwd(dnp.mean, dnp.quat, dnp.logscale, dnp.spectrum, qnp.x, qnp.n, qnp.wo,
                              gout, None, qnp.valid, mode=oracle.GPF_SUM, r_max=R, cutoff_sigma=3.0)
    for name in ("mean", "quat", "logscale", "spectrum"):
        assert grad_err(getattr(g, name).cpu().numpy(), ref[name]) <= GRAD_TOL, name


@pytest.mark.parametrize("mean32", [True, False])
def test_bf16_quantisation_error_against_the_float32_parameters(gpf, mean32):
    """What 16-bit storage costs: the radiance of the quantised field against
    the oracle on the float32 parameters it came from (8-bin spectrum).
    Float32 means: bfloat16 spectra alone allow a relative error of one unit
    roundoff, 2^-8, per term (hence per pixel), and the log-scale and
    rotation offsets add a little. Bfloat16 means (offsets of up to several
    scales, eight significant bits): errors of whole per cent, reported."""
    from paper_2512_12459_gb300.setup_index import make_index
    f = _field(60000, seed=66, channels=8)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 192, 160)
    queries = gpf.Queries.from_numpy(qnp)
    fb = gpf.Field.from_numpy(f).quantized(mean32=mean32)
    idx = make_index(fb, queries, query_cell=0.05)
    idx.build(fb, queries)
    o, _ = gpf.gpf_radiance_fwd(idx, fb, queries, gpf.GPF_SUM, r_max=R)
    sel = sample_active(qnp, 400, seed=67)
    ref = oracle_fwd(f, qnp, oracle.GPF_SUM, R, 3.0, sel)
    out = o.cpu().numpy().astype(np.float64)[:, sel]
    rel = np.abs(out - ref["out"]) / np.maximum(ref["denom"], 1e-20)
    keep = ~ref["near_cutoff"] & (ref["denom"].max(axis=0) > 0)
    per_pixel = rel[:, keep].max(axis=0)
    print(f"16-bit storage ({'float32' if mean32 else 'bfloat16'} means), per-pixel relative "
          f"error: median {np.median(per_pixel):.2e}, 99th percentile "
          f"{np.percentile(per_pixel, 99):.2e}, max {per_pixel.max():.2e}")
    if mean32:
        assert per_pixel.max() <= 2.0 ** -8 * 1.3
    else:
        assert np.median(per_pixel) <= 0.2


def test_train_step_with_bf16_store_replays_eager(gpf):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    from paper_2512_12459_gb300.train import TrainStep
    f = _field(20000, seed=68)
    qnp = synth.uneven_views(4, seed=69, sides=(32, 48))
    queries = gpf.Queries.from_numpy(qnp)
    tgt = synth.perturbed_copy(f, seed=70)
    tf = gpf.Field.from_numpy(tgt)
    ti = make_index(tf, queries, query_cell=0.05)
    ti.build(tf, queries)
    target = gpf.gpf_radiance_fwd(ti, tf, queries, gpf.GPF_SUM, r_max=R)[0].clone()
    steps = []
    for capture in (False, True):
        master = gpf.Field.from_numpy(f)
        store = master.quantized(mean32=True)
        idx = make_index(store, queries, query_cell=0.05, headroom=1.5)
        st = TrainStep(master, queries, target, idx, r_max=R, lr=5e-3, store=store)
        if capture:
            st.capture(warmup=1)
        else:
            st()
        losses = []
        for _ in range(5):
            st()
            losses.append(st.loss_value())
        steps.append((master, store, losses))
    (ma, sa, la), (mb, sb, lb) = steps
    assert la == lb and la[-1] < la[0]
    for x, y in zip(ma.tensors() + sa.tensors() + [sa.anchor], mb.tensors() + sb.tensors() + [sb.anchor]):
        assert torch.equal(x, y)
