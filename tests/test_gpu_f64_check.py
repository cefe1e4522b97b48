"""The float64 gradient-check build of the backward (gpf_query_params.f64_sums):
the same float32 pair terms as the product path, summed, reduced and turned
into gradients in float64. Against the FP64 oracle (whose gradients are
pinned by central finite differences) it must agree to 1e-6 normwise per
gradient tensor, where float32 summation order can no longer hide a wrong
term (Sec. 4.2, Differentiable Accumulation). Hit points that have a pair
within 1e-4 of the cutoff (which float32 and float64 may classify
differently) get a zero upstream gradient, which removes every contribution
they make. In GPF_NORMALIZED mode the backward is given the oracle's forward
(rounded to float32) as its `out` and `z`, so that the check covers the
backward alone."""

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import GRAD_TOL, INF, grad_err

pytestmark = pytest.mark.gpu

KEYS = ("mean", "quat", "logscale", "spectrum")
F64_TOL = 1e-6
GAPS = []


@pytest.fixture(scope="module")
def gpf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12459_gb300 as g
    return g


def _check(gpf, fnp, qnp, mode, r_max, cutoff, cell=0.1, brute=False, seed=0):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((fnp.channels, qnp.m))
    fo = oracle.radiance_fwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, qnp.x, qnp.n,
                             qnp.wo, qnp.albedo, qnp.valid, mode=mode, r_max=r_max,
                             cutoff_sigma=cutoff)
    G[:, fo["near_cutoff"]] = 0.0
    G = G.astype(np.float32)
    ref = oracle.radiance_bwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, qnp.x, qnp.n,
                              qnp.wo, G, qnp.albedo, qnp.valid, mode=mode, r_max=r_max,
                              cutoff_sigma=cutoff)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=cell, cutoff_sigma=cutoff, brute_force=brute)
    idx.build(field, queries)
    out = torch.as_tensor(fo["out"], dtype=torch.float32, device="cuda").contiguous()
    z = torch.as_tensor(fo["Z"], dtype=torch.float32, device="cuda").contiguous()
    Gt = torch.as_tensor(G, device="cuda")
    res = {}
    for f64 in (True, False):
        g = gpf.gpf_radiance_bwd(idx, field, queries, Gt, out, z, mode, r_max=r_max,
                                 f64_sums=f64)
        torch.cuda.synchronize()
        res[f64] = {k: grad_err(getattr(g, k).cpu().numpy().astype(np.float64), ref[k])
                    for k in KEYS}
    GAPS.append((mode, r_max, cutoff, res[True], res[False]))
    for k in KEYS:
        assert res[True][k] < F64_TOL, ("float64 sums", k, res[True])
        assert res[False][k] < GRAD_TOL, ("float32 sums", k, res[False])
    return res


@pytest.mark.parametrize("mode", [oracle.GPF_SUM, oracle.GPF_NORMALIZED])
@pytest.mark.parametrize("r_max", [INF, 0.05])
def test_f64_sums_brute_force(gpf, mode, r_max):
    fnp, qnp = synth.config1_random(seed=50, n=300, m=3000 + 11, albedo=True)
    _check(gpf, fnp, qnp, mode, r_max, INF)


@pytest.mark.parametrize("mode", [oracle.GPF_SUM, oracle.GPF_NORMALIZED])
def test_f64_sums_culled(gpf, mode):
    fnp, qnp = synth.config1_random(seed=51, n=600, m=6000 + 7, albedo=True)
    _check(gpf, fnp, qnp, mode, 0.05, 3.0, cell=0.1)


@pytest.mark.parametrize("mode", [oracle.GPF_SUM, oracle.GPF_NORMALIZED])
def test_f64_sums_caustic_scene(gpf, mode):
    pos, flux = synth.caustic_photons(3000, seed=52)
    fnp = synth.field_from_photons(pos, flux, seed=52)
    rng = np.random.default_rng(52)
    fnp.logscale = (fnp.logscale + rng.normal(0.0, 0.3, fnp.logscale.shape)).astype(np.float32)
    qnp = synth.pinhole_hitpoints((0.0, -6.0, 4.0), (0.0, 0.0, 0.5), 72, 64)
    _check(gpf, fnp, qnp, mode, 0.02, 3.0, cell=0.05)


def test_report_f32_f64_gap():
    """Prints the normwise errors of both builds (after the cases above)."""
    for mode, r, cut, e64, e32 in GAPS:
        print(f"mode {mode} r {r} cutoff {cut}: f64 " +
              ", ".join(f"{k} {e64[k]:.1e}" for k in KEYS) + " | f32 " +
              ", ".join(f"{k} {e32[k]:.1e}" for k in KEYS))
