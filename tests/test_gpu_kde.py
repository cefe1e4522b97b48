"""The per-view photon density estimate (GPF_DISK_KDE, Sec. 3.2 Eq. kde) on
the GPU against the oracle: exact lattice counts and a caustic photon map."""

import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12459_gb300 as g
    return g


def _kde(gpf, pos, flux, qnp, radius, cell, split_items=0):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    field = gpf.photon_field(torch.as_tensor(pos, dtype=torch.float32, device="cuda"),
                             torch.as_tensor(flux, dtype=torch.float32, device="cuda"), radius)
    queries = gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=cell, split_items=split_items)
    idx.build(field, queries)
    out, z = gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_DISK_KDE, r_max=radius)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), z.cpu().numpy(), (idx, field, queries, out, z)


@pytest.mark.parametrize("R", [5.0, 2.5, 1.0])
def test_lattice_counts_are_exact(gpf, R):
    """Photons on a lattice of spacing 2^-4 (exact in float32): every hit
    point on or between lattice points gathers exactly the photons with
    |d| <= R h, the edge included."""
    h = 0.0625
    ij = np.array([(i, j) for i in range(-12, 13) for j in range(-12, 13)], np.float64)
    pos = np.zeros((3, len(ij)))
    pos[:2] = ij.T * h
    flux = np.stack([np.ones(len(ij)), np.arange(len(ij)) % 7 + 1.0])
    qx = np.array([(a * h, b * h) for a in range(-4, 5) for b in range(-4, 5)] +
                  [(a * h + h / 2, b * h) for a in range(-3, 3) for b in range(-3, 3)], np.float64)
    m = len(qx)
    qnp = synth.Queries(x=np.vstack([qx.T, np.zeros(m)]).astype(np.float32),
                        n=np.tile([[0.0], [0.0], [1.0]], (1, m)).astype(np.float32),
                        wo=np.tile([[0.0], [0.0], [1.0]], (1, m)).astype(np.float32),
                        valid=np.ones(m, np.uint8))
    out, z, _ = _kde(gpf, pos.astype(np.float32), flux.astype(np.float32), qnp, R * h, 0.1)
    ref = oracle.disk_kde(pos, flux, qnp.x, qnp.n, qnp.wo, R * h)
    assert np.array_equal(z, ref["count"].astype(np.float32))
    np.testing.assert_allclose(out, ref["out"], rtol=2e-7, atol=0)


@pytest.mark.parametrize("radius,split", [(0.02, 0), (0.05, 0), (0.02, 256)])
def test_caustic_photon_map_matches_the_oracle(gpf, radius, split):
    """split > 0: the dense tiles' lists split over several work units."""
    pos, flux = synth.caustic_photons(60000, seed=81)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 160, 128)
    out, z, _ = _kde(gpf, pos.T, flux.T, qnp, radius, 0.05, split)
    from gpu_helpers import sample_active
    sel = sample_active(qnp, 500, seed=82)
    ref = oracle.disk_kde(pos.T, flux.T, qnp.x[:, sel], qnp.n[:, sel], qnp.wo[:, sel], radius,
                          valid=qnp.valid[sel])
    keep = ~ref["near"]
    assert keep.sum() > 0.9 * len(sel) and ref["count"][keep].max() > 20
    err = np.abs(out[:, sel] - ref["out"]) / np.maximum(ref["denom"], 1e-30)
    assert err[:, keep].max() <= 1e-5
    assert np.array_equal(z[sel][keep], ref["count"][keep].astype(np.float32))
    # points where nothing is gathered return exactly zero
    assert np.all(out[:, sel][:, ref["count"] == 0] == 0)


def test_no_gradient_for_the_density_estimate(gpf):
    import torch
    pos, flux = synth.caustic_photons(2000, seed=83)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 32, 24)
    out, z, (idx, field, queries, o, zz) = _kde(gpf, pos.T, flux.T, qnp, 0.05, 0.1)
    with pytest.raises(gpf.GPFError):
        gpf.gpf_radiance_bwd(idx, field, queries, torch.ones_like(o), o, zz, gpf.GPF_DISK_KDE,
                             r_max=0.05)
    assert math.isfinite(float(out.sum()))
