"""Pins the FP64 oracle to things other than itself: hand-derived closed forms,
Gaussian integrals, a library multivariate-normal density, a separately
written kernel density estimate, invariances, finite differences and
torch.optim.Adam. CPU only."""

import math
import zlib

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.stats import chi2, multivariate_normal, norm

import oracle
import synth
from golden_util import load_constants, load_examples


def _fwd(f, q, **kw):
    return oracle.radiance_fwd(f["mean"], f["quat"], f["logscale"], f["spectrum"],
                               q["x"], q["n"], q["wo"], **kw)


def _sigma_from_library(quat_wxyz, scale):
    """Covariance R S S^T R^T with R from scipy (scalar-last quaternion)."""
    w, x, y, z = quat_wxyz
    R = Rotation.from_quat([x, y, z, w]).as_matrix()
    return R @ np.diag(np.asarray(scale) ** 2) @ R.T


def _rand_field(rng, n, c=3, spread=1.0, lmean=-2.0, lstd=0.4):
    q = rng.standard_normal((4, n))
    return {"mean": rng.uniform(0, spread, (3, n)), "quat": q,
            "logscale": rng.normal(lmean, lstd, (3, n)), "spectrum": rng.uniform(0.1, 1.0, (c, n))}


def _facing(m):
    n = np.zeros((3, m)); n[2] = 1.0
    return n, n.copy()


# --------------------------------------------------------------------------- worked examples

def test_worked_examples_closed_forms():
    examples, _ = load_examples()
    for name, ex in examples.items():
        res = oracle.radiance_fwd(ex["mean"], ex["quat"], ex["logscale"], ex["spectrum"],
                                  ex["x"], ex["n"], ex["wo"], albedo=ex["albedo"],
                                  mode=ex["mode"], r_max=ex["r_max"],
                                  cutoff_sigma=ex["cutoff_sigma"])
        # inputs are rounded to float32, so the closed form holds to ~1e-6
        np.testing.assert_allclose(res["out"], ex["expected"], rtol=2e-6, atol=1e-12,
                                   err_msg=name)


def test_worked_gradient_closed_forms():
    examples, grads = load_examples()
    for name, g in grads.items():
        ex = examples[g["example"]]
        res = oracle.radiance_bwd(ex["mean"], ex["quat"], ex["logscale"], ex["spectrum"],
                                  ex["x"], ex["n"], ex["wo"], g["grad_out"], albedo=ex["albedo"],
                                  mode=ex["mode"], r_max=ex["r_max"],
                                  cutoff_sigma=ex["cutoff_sigma"])
        for k, exp in g["expected"].items():
            np.testing.assert_allclose(res[k], exp, rtol=5e-6, atol=1e-7, err_msg=f"{name}:{k}")


def test_paper_constants_fixture():
    c = load_constants()
    assert c["query_radius_r"] == 0.02 and c["normalisation_eps"] == 1e-6
    assert c["adam_lr"] == 5e-4 and c["k_min"] == 3


# --------------------------------------------------------------------------- weight vs library density

def test_single_gaussian_weight_is_scaled_normal_density():
    """w(x) = (2 pi)^{3/2} sqrt(det Sigma) N(x; mu, Sigma) with Sigma built by scipy's
    quaternion convention; catches a transposed R, a wrong quaternion order or a
    scale used as a variance."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        q = rng.standard_normal(4)
        s = np.exp(rng.normal(-2, 0.7, 3))
        mu = rng.uniform(-1, 1, 3)
        x = mu + rng.normal(0, 1.5 * s.max(), (5, 3))
        f = {"mean": mu[:, None], "quat": q[:, None], "logscale": np.log(s)[:, None],
             "spectrum": np.ones((1, 1))}
        n, wo = _facing(5)
        res = _fwd(f, {"x": x.T, "n": n, "wo": wo}, cutoff_sigma=math.inf)
        Sig = _sigma_from_library(q / np.linalg.norm(q), s)
        ref = (2 * np.pi) ** 1.5 * np.sqrt(np.linalg.det(Sig)) * \
            multivariate_normal(mean=mu, cov=Sig).pdf(x)
        np.testing.assert_allclose(res["out"][0], ref, rtol=1e-9, atol=1e-300)


# --------------------------------------------------------------------------- integrals (P1, P2)

def _grid3(center, half, k):
    ax = [np.linspace(c - half, c + half, k) for c in center]
    h = ax[0][1] - ax[0][0]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()]), h ** 3


@pytest.mark.parametrize("cutoff,factor,rtol", [(math.inf, 1.0, 1e-8),
                                               (3.0, chi2.cdf(9.0, 3), 3e-3)])
def test_volume_integral_of_one_gaussian(cutoff, factor, rtol):
    """Integral over R^3 of w = (2 pi)^{3/2} s1 s2 s3 (the unnormalised form of
    the unit 3D integral the paper contrasts with surfaces, Sec. 2); truncated
    to Q <= 9 it is scaled by P(chi^2_3 <= 9) = 0.970709."""
    q = np.array([0.8, -0.3, 0.5, 0.2])
    s = np.array([0.12, 0.07, 0.05])
    mu = np.array([0.3, -0.2, 0.1])
    half = (6.0 if math.isinf(cutoff) else 3.05) * s.max()
    k = 121 if math.isinf(cutoff) else 161
    X, dv = _grid3(mu, half, k)
    f = {"mean": mu[:, None], "quat": q[:, None], "logscale": np.log(s)[:, None],
         "spectrum": np.ones((1, 1))}
    n, wo = _facing(X.shape[1])
    res = _fwd(f, {"x": X, "n": n, "wo": wo}, cutoff_sigma=cutoff)
    integral = res["out"][0].sum() * dv
    exact = (2 * np.pi) ** 1.5 * np.prod(s) * factor
    assert abs(integral / exact - 1.0) < rtol


def test_plane_integral_depends_on_orientation():
    """Over a plane through mu with unit normal n: integral of w dA =
    2 pi s1 s2 s3 / sqrt(n^T Sigma n) (the surface integral of a 3D Gaussian
    depends on the surface's pose, Sec. 2)."""
    rng = np.random.default_rng(3)
    for _ in range(4):
        q = rng.standard_normal(4)
        s = np.exp(rng.normal(-2.3, 0.5, 3))
        mu = rng.uniform(-0.5, 0.5, 3)
        nrm = rng.standard_normal(3); nrm /= np.linalg.norm(nrm)
        t1 = np.cross(nrm, [1.0, 0.0, 0.0] if abs(nrm[0]) < 0.9 else [0.0, 1.0, 0.0])
        t1 /= np.linalg.norm(t1)
        t2 = np.cross(nrm, t1)
        half, k = 7.0 * s.max(), 401
        a = np.linspace(-half, half, k)
        A, B = np.meshgrid(a, a, indexing="ij")
        X = mu[:, None] + t1[:, None] * A.ravel() + t2[:, None] * B.ravel()
        f = {"mean": mu[:, None], "quat": q[:, None], "logscale": np.log(s)[:, None],
             "spectrum": np.ones((1, 1))}
        n, wo = _facing(X.shape[1])
        res = _fwd(f, {"x": X, "n": n, "wo": wo}, cutoff_sigma=math.inf)
        integral = res["out"][0].sum() * (a[1] - a[0]) ** 2
        Sig = _sigma_from_library(q / np.linalg.norm(q), s)
        exact = 2 * np.pi * np.prod(s) / np.sqrt(nrm @ Sig @ nrm)
        assert abs(integral / exact - 1.0) < 1e-7


# --------------------------------------------------------------------------- isotropic collapse (P3)

def _kde2d(points, weights, h, xq):
    """Weighted 2D Gaussian-kernel density estimate with bandwidth h (a kernel
    density estimate as in the photon density estimate of Sec. 3.2, with a
    smooth kernel in place of the disk): sum_i W_i N(x; p_i, h^2 I)."""
    out = np.zeros(xq.shape[0])
    for p, wgt in zip(points, weights):
        out += wgt * norm.pdf(xq[:, 0], p[0], h) * norm.pdf(xq[:, 1], p[1], h)
    return out


def test_isotropic_field_on_a_plane_is_a_kde():
    rng = np.random.default_rng(5)
    n, m, h = 60, 80, 0.07
    mu = np.zeros((3, n)); mu[:2] = rng.uniform(0, 1, (2, n))
    spec = rng.uniform(0.1, 1.0, (3, n))
    f = {"mean": mu, "quat": rng.standard_normal((4, n)),
         "logscale": np.full((3, n), np.log(h)), "spectrum": spec}
    x = np.zeros((3, m)); x[:2] = rng.uniform(0, 1, (2, m))
    nn, wo = _facing(m)
    res = _fwd(f, {"x": x, "n": nn, "wo": wo}, cutoff_sigma=math.inf)
    for c in range(3):
        ref = 2 * np.pi * h * h * _kde2d(mu[:2].T, spec[c], h, x[:2].T)
        np.testing.assert_allclose(res["out"][c], ref, rtol=1e-10)


# --------------------------------------------------------------------------- invariances (P4, P5, P7)

def test_isotropic_gaussian_ignores_rotation():
    rng = np.random.default_rng(8)
    n, m = 40, 50
    f = _rand_field(rng, n)
    f["logscale"] = np.tile(rng.normal(-2.5, 0.3, n), (3, 1))
    x = rng.uniform(0, 1, (3, m)); nn, wo = _facing(m)
    a = _fwd(f, {"x": x, "n": nn, "wo": wo}, r_max=0.1, cutoff_sigma=3.0)
    f2 = dict(f); f2["quat"] = rng.standard_normal((4, n))
    b = _fwd(f2, {"x": x, "n": nn, "wo": wo}, r_max=0.1, cutoff_sigma=3.0)
    np.testing.assert_allclose(a["out"], b["out"], rtol=1e-11, atol=1e-300)


def test_normalized_single_contributor_returns_its_flux():
    rng = np.random.default_rng(9)
    f = _rand_field(rng, 1)
    x = f["mean"] + rng.normal(0, 0.05, (3, 7)); nn, wo = _facing(7)
    res = _fwd(f, {"x": x, "n": nn, "wo": wo}, mode=oracle.GPF_NORMALIZED,
               cutoff_sigma=math.inf)
    big = res["Z"] > 1e-6
    assert big.sum() >= 3
    np.testing.assert_allclose(res["out"][:, big], np.repeat(f["spectrum"], big.sum(), 1),
                               rtol=1e-12)


def test_normalized_constant_flux_returns_it():
    rng = np.random.default_rng(10)
    f = _rand_field(rng, 30, spread=0.3)
    f["spectrum"] = np.tile(np.array([[0.3], [1.7], [2.2]]), (1, 30))
    x = rng.uniform(0, 0.3, (3, 25)); nn, wo = _facing(25)
    res = _fwd(f, {"x": x, "n": nn, "wo": wo}, mode=oracle.GPF_NORMALIZED,
               cutoff_sigma=math.inf)
    big = res["Z"] > 1e-6
    np.testing.assert_allclose(res["out"][:, big],
                               np.tile([[0.3], [1.7], [2.2]], (1, big.sum())), rtol=1e-12)


def test_permutation_and_translation_invariance():
    rng = np.random.default_rng(12)
    n, m = 50, 40
    f = _rand_field(rng, n)
    x = rng.uniform(0, 1, (3, m)); nn, wo = _facing(m)
    kw = dict(r_max=0.08, cutoff_sigma=3.0)
    a = _fwd(f, {"x": x, "n": nn, "wo": wo}, **kw)
    p = rng.permutation(n)
    fp = {k: v[:, p] for k, v in f.items()}
    b = _fwd(fp, {"x": x, "n": nn, "wo": wo}, **kw)
    np.testing.assert_allclose(a["out"], b["out"], rtol=1e-12, atol=1e-300)
    shift = np.array([[0.25], [-0.5], [1.0]])     # exactly representable shift
    ft = dict(f); ft["mean"] = f["mean"] + shift
    c = _fwd(ft, {"x": x + shift, "n": nn, "wo": wo}, **kw)
    np.testing.assert_allclose(a["out"], c["out"], rtol=1e-9, atol=1e-300)


def test_hemisphere_gate_and_valid_mask():
    rng = np.random.default_rng(13)
    f = _rand_field(rng, 20, spread=0.2)
    m = 30
    x = rng.uniform(0, 0.2, (3, m))
    nn = rng.standard_normal((3, m)); wo = rng.standard_normal((3, m))
    valid = (rng.uniform(0, 1, m) < 0.7).astype(np.uint8)
    res = _fwd(f, {"x": x, "n": nn, "wo": wo}, valid=valid, cutoff_sigma=math.inf)
    facing = np.sum(nn * wo, axis=0) > 0
    on = facing & valid.astype(bool)
    assert np.all(res["out"][:, ~on] == 0.0)
    assert np.all(res["out"][:, on] > 0.0)


# --------------------------------------------------------------------------- falloff psi

def test_falloff_special_values():
    r = 0.02
    assert oracle.falloff_psi(np.array([0.0, r / 2, r]), r).tolist() == [1.0, 1.0, 1.0]
    np.testing.assert_allclose(oracle.falloff_psi(np.array([2 * r]), r), [math.exp(-3.0)],
                               rtol=1e-14)
    np.testing.assert_allclose(oracle.falloff_psi(np.array([r * (1 + 1 / math.sqrt(3))]), r),
                               [math.exp(-1.0)], rtol=1e-14)
    d = np.linspace(0, 5 * r, 1001)
    p = oracle.falloff_psi(d, r)
    assert np.all(np.diff(p) <= 0.0)
    assert abs(oracle.falloff_psi(np.array([r * (1 + 1e-9)]), r)[0] - 1.0) < 1e-15
    assert np.all(oracle.falloff_psi(d, math.inf) == 1.0)


def test_falloff_uses_euclidean_distance():
    """Anisotropic Gaussian, point 2r away along the long local axis: the
    falloff sees the Euclidean distance (t = 1, psi = e^-3) and the Gaussian
    sees the Mahalanobis one."""
    r = 0.02
    q = np.array([math.cos(math.pi / 8), 0, 0, math.sin(math.pi / 8)])
    s = np.array([0.5, 0.01, 0.01])
    axis = np.array([math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0])
    x = (2 * r * axis)[:, None]
    f = {"mean": np.zeros((3, 1)), "quat": q[:, None], "logscale": np.log(s)[:, None],
         "spectrum": np.ones((1, 1))}
    nn, wo = _facing(1)
    res = _fwd(f, {"x": x, "n": nn, "wo": wo}, r_max=r, cutoff_sigma=math.inf)
    exact = math.exp(-0.5 * (2 * r / 0.5) ** 2) * math.exp(-3.0)
    np.testing.assert_allclose(res["out"][0, 0], exact, rtol=1e-12)


# --------------------------------------------------------------------------- gradients (P8)

def _objective(f, q, G, kw):
    out = oracle.radiance_fwd(f["mean"], f["quat"], f["logscale"], f["spectrum"],
                              q["x"], q["n"], q["wo"], albedo=q.get("albedo"), **kw)["out"]
    return float(np.sum(G * out))


def _fd(f, q, G, kw, key, h):
    g = np.zeros_like(f[key])
    for idx in np.ndindex(*f[key].shape):
        fp = {k: v.copy() for k, v in f.items()}
        fm = {k: v.copy() for k, v in f.items()}
        fp[key][idx] += h
        fm[key][idx] -= h
        g[idx] = (_objective(fp, q, G, kw) - _objective(fm, q, G, kw)) / (2 * h)
    return g


FD_CASES = [
    ("sum_plain", dict(mode=oracle.GPF_SUM, r_max=math.inf, cutoff_sigma=math.inf)),
    ("sum_falloff", dict(mode=oracle.GPF_SUM, r_max=0.06, cutoff_sigma=math.inf)),
    ("sum_cutoff", dict(mode=oracle.GPF_SUM, r_max=0.06, cutoff_sigma=3.0)),
    ("norm_plain", dict(mode=oracle.GPF_NORMALIZED, r_max=math.inf, cutoff_sigma=math.inf)),
    ("norm_falloff_cutoff", dict(mode=oracle.GPF_NORMALIZED, r_max=0.05, cutoff_sigma=3.0)),
]


@pytest.mark.parametrize("name,kw", FD_CASES, ids=[c[0] for c in FD_CASES])
def test_analytic_gradient_matches_central_differences(name, kw):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    n, m, c = 5, 36, 3
    f = {"mean": rng.uniform(0, 0.25, (3, n)), "quat": rng.standard_normal((4, n)),
         "logscale": rng.normal(-2.2, 0.3, (3, n)), "spectrum": rng.uniform(-0.5, 1.0, (c, n))}
    x = rng.uniform(-0.05, 0.3, (3, m))
    nn = rng.standard_normal((3, m)); wo = rng.standard_normal((3, m))
    q = {"x": x, "n": nn, "wo": wo, "albedo": rng.uniform(0.3, 1.0, (c, m))}
    G = rng.standard_normal((c, m))
    fwd = oracle.radiance_fwd(f["mean"], f["quat"], f["logscale"], f["spectrum"], x, nn, wo,
                              albedo=q["albedo"], band=1e-2, **kw)
    if math.isfinite(kw["cutoff_sigma"]):
        assert not fwd["near_cutoff"].any(), "FD point too close to the cutoff"
    if kw["mode"] == oracle.GPF_NORMALIZED:
        assert np.all(np.abs(fwd["Z"] - 1e-6) > 1e-8)
    an = oracle.radiance_bwd(f["mean"], f["quat"], f["logscale"], f["spectrum"], x, nn, wo, G,
                             albedo=q["albedo"], **kw)
    for key, h in (("mean", 1e-6), ("quat", 1e-6), ("logscale", 1e-6), ("spectrum", 1e-6)):
        num = _fd(f, q, G, kw, key, h)
        err = np.linalg.norm(num - an[key]) / max(np.linalg.norm(an[key]), 1e-300)
        assert err < 1e-6, (name, key, err)
        assert np.linalg.norm(an[key]) > 0.0


def test_gradient_of_the_worked_example_by_differences():
    examples, grads = load_examples()
    g = grads["axis_aligned_single_grad"]
    ex = examples[g["example"]]
    f = {k: ex[k].astype(np.float64) for k in ("mean", "quat", "logscale", "spectrum")}
    q = {"x": ex["x"], "n": ex["n"], "wo": ex["wo"]}
    kw = dict(mode=ex["mode"], r_max=ex["r_max"], cutoff_sigma=ex["cutoff_sigma"])
    for key, exp in g["expected"].items():
        num = _fd(f, q, g["grad_out"], kw, key, 1e-7)
        np.testing.assert_allclose(num, exp, rtol=1e-5, atol=1e-7)


# --------------------------------------------------------------------------- loss and Adam (P10)

def test_mse_loss_and_gradient():
    rng = np.random.default_rng(21)
    O = rng.standard_normal((3, 40)); T = rng.standard_normal((3, 40))
    valid = (rng.uniform(0, 1, 40) < 0.6).astype(np.uint8)
    nv = valid.sum()
    ref = sum(np.sum((O[:, i] - T[:, i]) ** 2) for i in range(40) if valid[i]) / nv
    assert abs(oracle.mse_loss(O, T, valid) - ref) < 1e-12
    g = oracle.mse_loss_grad(O, T, valid)
    h = 1e-6
    for idx in [(0, 0), (1, 5), (2, 17), (0, 33)]:
        Op, Om = O.copy(), O.copy()
        Op[idx] += h; Om[idx] -= h
        num = (oracle.mse_loss(Op, T, valid) - oracle.mse_loss(Om, T, valid)) / (2 * h)
        assert abs(num - g[idx]) < 1e-7
    assert oracle.mse_loss(O, T, np.zeros(40, np.uint8)) == 0.0


def test_adam_matches_torch_optim_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(22)
    p0 = rng.standard_normal(257)
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=5e-4, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(257), np.zeros(257)
    for step in range(1, 201):
        g = rng.standard_normal(257) * (1.0 + step % 7)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = oracle.adam_step(p, g, m, v, step, lr=5e-4)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=0, atol=1e-12)


# --------------------------------------------------------------------------- planted mistakes

def _expect_failure(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return
    raise AssertionError(f"{fn.__name__} did not notice the planted mistake")


def test_pins_catch_a_transposed_rotation(monkeypatch):
    import oracle.gpf_oracle as go
    good = go.quat_to_rotmat
    monkeypatch.setattr(go, "quat_to_rotmat", lambda q: np.swapaxes(good(q), -1, -2))
    _expect_failure(test_single_gaussian_weight_is_scaled_normal_density)
    _expect_failure(test_worked_examples_closed_forms)
    _expect_failure(test_plane_integral_depends_on_orientation)


def test_pins_catch_falloff_on_the_wrong_distance(monkeypatch):
    import oracle.gpf_oracle as go
    good = go.falloff_psi
    monkeypatch.setattr(go, "falloff_psi", lambda d, r: good(d * d / max(r, 1e-6), r))
    _expect_failure(test_falloff_uses_euclidean_distance)
    _expect_failure(test_worked_examples_closed_forms)


def test_pins_catch_a_wrong_gradient_term(monkeypatch):
    import oracle.gpf_oracle as go
    good = go._falloff_dpsi_ddist
    monkeypatch.setattr(go, "_falloff_dpsi_ddist", lambda d, r: -good(d, r))
    _expect_failure(test_analytic_gradient_matches_central_differences, *FD_CASES[1])
    monkeypatch.setattr(go, "_falloff_dpsi_ddist", good)
    goodp = go._rotmat_partials
    def swapped(qh):
        P = goodp(qh)
        return P[:, [0, 2, 1, 3]]
    monkeypatch.setattr(go, "_rotmat_partials", swapped)
    _expect_failure(test_analytic_gradient_matches_central_differences, *FD_CASES[0])
    _expect_failure(test_worked_gradient_closed_forms)


def test_pins_catch_a_wrong_cutoff(monkeypatch):
    import oracle.gpf_oracle as go
    good = go._pairs
    monkeypatch.setattr(go, "_pairs", lambda P, xs, r, c: good(P, xs, r, c * c if math.isfinite(c) else c))
    _expect_failure(test_volume_integral_of_one_gaussian, 3.0, chi2.cdf(9.0, 3), 3e-3)
    _expect_failure(test_worked_examples_closed_forms)


# ---- the photon density estimate (Sec. 3.2, Eq. kde)

def _lattice(h, half, flux=1.0):
    ij = np.array([(i, j) for i in range(-half, half + 1) for j in range(-half, half + 1)], float)
    pos = np.zeros((3, len(ij)))
    pos[:2] = ij.T * h
    return pos, np.full((1, len(ij)), flux)


def _gauss_circle(radius_in_cells):
    """Lattice points (i, j) with i^2 + j^2 <= R^2, by integer enumeration."""
    R2 = radius_in_cells ** 2
    k = int(np.floor(radius_in_cells)) + 1
    return sum(1 for i in range(-k, k + 1) for j in range(-k, k + 1) if i * i + j * j <= R2)


@pytest.mark.parametrize("R,count", [(5.0, 81), (2.5, 21), (1.0, 5), (0.5, 1)])
def test_disk_kde_counts_lattice_photons(R, count):
    """Photons on a square lattice (spacing h, unit flux), gathered at a
    lattice point with radius R h: the Gauss circle count, edge included
    (R = 5 puts (3, 4) and (5, 0) on the edge), over the disk area."""
    h = 0.25
    pos, flux = _lattice(h, 8)
    assert _gauss_circle(R) == count
    x = np.zeros((3, 1))
    n = np.array([[0.0], [0.0], [1.0]])
    out = oracle.disk_kde(pos, flux, x, n, n, R * h)
    np.testing.assert_allclose(out["out"][0, 0], count / (np.pi * (R * h) ** 2), rtol=1e-14)
    assert out["count"][0] == count


def test_disk_kde_single_photon_gate_and_albedo():
    pos = np.array([[0.1], [0.0], [0.0]])
    flux = np.array([[2.0], [4.0]])
    x = np.array([[0.0, 0.0, 0.0, 0.5], [0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0]])
    n = np.array([[0.0] * 4, [0.0] * 4, [1.0] * 4])
    wo = n.copy()
    wo[2, 1] = -1.0                                  # facing away
    alb = np.array([[0.5] * 4, [0.25] * 4])
    valid = np.array([1, 1, 0, 1], np.uint8)
    out = oracle.disk_kde(pos, flux, x, n, wo, 0.2, albedo=alb, valid=valid)["out"]
    a = np.pi * 0.04
    np.testing.assert_allclose(out[:, 0], [0.5 * 2 / a, 0.25 * 4 / a], rtol=1e-14)
    assert np.all(out[:, 1:] == 0)                   # gate, invalid, out of reach


# ---- the hybrid neighbourhood (Sec. 4.2, Neighborhood Search; Algorithm S3)

def _line_field(dists, phis, s=0.02):
    """Isotropic Gaussians on the x axis at the given distances from the origin."""
    n = len(dists)
    mean = np.zeros((3, n))
    mean[0] = dists
    quat = np.zeros((4, n))
    quat[0] = 1.0
    return mean, quat, np.full((3, n), np.log(s)), np.array([phis], float)


def _w_line(d, s=0.02, r=0.02):
    """exp(-d^2 / (2 s^2)) psi(d) for a Gaussian at distance d on the axis."""
    psi = 1.0 if d <= r else math.exp(-3.0 * ((d - r) / r) ** 2)
    return math.exp(-0.5 * (d / s) ** 2) * psi


@pytest.mark.parametrize("ball_r,k_min,members", [
    (0.02, 3, [0, 1, 2]),        # one mean in the ball, fewer than 3: the 3 nearest
    (0.06, 3, [0, 1, 2]),        # exactly 3 in the ball: the ball
    (0.08, 3, [0, 1, 2, 3]),     # 4 in the ball: the ball
    (0.02, 0, [0]),              # ball only (Table 3, w_radius)
    (0.0, 2, [0, 1]),            # kNN only (Table 3, w_knn)
    (0.005, 0, []),              # empty ball, no kNN: nothing
])
def test_hybrid_neighbourhood_selects_the_paper_sets(ball_r, k_min, members):
    dists = [0.01, 0.03, 0.05, 0.07, 0.2]
    phis = [1.0, 2.0, 4.0, 8.0, 16.0]
    mean, quat, lsc, spec = _line_field(dists, phis)
    x = np.zeros((3, 1))
    nrm = np.array([[0.0], [0.0], [1.0]])
    for mode in (oracle.GPF_SUM, oracle.GPF_NORMALIZED):
        out = oracle.hybrid_fwd(mean, quat, lsc, spec, x, nrm, nrm, mode=mode, r_max=0.02,
                                ball_r=ball_r, k_min=k_min)
        L = sum(_w_line(dists[i]) * phis[i] for i in members)
        Z = sum(_w_line(dists[i]) for i in members)
        want = L if mode == oracle.GPF_SUM else L / max(Z, 1e-6)
        np.testing.assert_allclose(out["out"][0, 0], want, rtol=1e-13, atol=1e-300)
        assert out["n_nb"][0] == len(members)


def test_hybrid_knn_ties_go_to_the_smaller_index():
    # Gaussians 1 and 2 at the same distance: with k_min = 2 the pair {0, 1}
    mean, quat, lsc, spec = _line_field([0.01, 0.05, -0.05], [1.0, 2.0, 4.0])
    x = np.zeros((3, 1))
    nrm = np.array([[0.0], [0.0], [1.0]])
    out = oracle.hybrid_fwd(mean, quat, lsc, spec, x, nrm, nrm, mode=oracle.GPF_SUM,
                            r_max=0.02, ball_r=0.02, k_min=2)
    want = _w_line(0.01) * 1.0 + _w_line(0.05) * 2.0
    np.testing.assert_allclose(out["out"][0, 0], want, rtol=1e-13)
    assert out["knn"][0] and out["near"][0]          # a tie is flagged as sensitive


def test_hybrid_with_a_ball_holding_everything_is_the_untruncated_sum():
    fnp, qnp = synth.config1_random(seed=33, n=60, m=40)
    a = oracle.hybrid_fwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, qnp.x, qnp.n, qnp.wo,
                          mode=oracle.GPF_NORMALIZED, r_max=0.05, ball_r=10.0, k_min=3)
    b = oracle.radiance_fwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, qnp.x, qnp.n,
                            qnp.wo, mode=oracle.GPF_NORMALIZED, r_max=0.05,
                            cutoff_sigma=math.inf)
    np.testing.assert_allclose(a["out"], b["out"], rtol=1e-12, atol=1e-300)


def _hybrid_objective(f, q, G, kw):
    out = oracle.hybrid_fwd(f["mean"], f["quat"], f["logscale"], f["spectrum"], q["x"], q["n"],
                            q["wo"], albedo=q.get("albedo"), **kw)["out"]
    return float(np.sum(G * out))


@pytest.mark.parametrize("mode", [oracle.GPF_SUM, oracle.GPF_NORMALIZED])
@pytest.mark.parametrize("ball_r,k_min", [(0.09, 3), (0.0, 4), (0.12, 0)])
def test_hybrid_gradient_matches_central_differences(mode, ball_r, k_min):
    """hybrid_bwd against central differences of hybrid_fwd. The selection
    N(x) is piecewise constant: the points are chosen so that no mean lies
    within 1e-3 (relative, in squared distance) of a ball's edge and no k-th /
    (k+1)-th nearest distances are that close, so steps of 1e-6 never change
    it and the differences see the smooth part only."""
    rng = np.random.default_rng(int(ball_r * 1000) * 31 + k_min * 7 + mode)
    n, m, c = 7, 24, 3
    f = {"mean": rng.uniform(0, 0.25, (3, n)), "quat": rng.standard_normal((4, n)),
         "logscale": rng.normal(-2.4, 0.3, (3, n)), "spectrum": rng.uniform(-0.5, 1.0, (c, n))}
    x = rng.uniform(0.0, 0.25, (3, m))
    nn = rng.standard_normal((3, m)); wo = rng.standard_normal((3, m))
    kw = dict(mode=mode, r_max=0.05, ball_r=ball_r, k_min=k_min)
    fwd = oracle.hybrid_fwd(f["mean"], f["quat"], f["logscale"], f["spectrum"], x, nn, wo,
                            band=1e-3, **kw)
    keep = ~fwd["near"]
    x, nn, wo = x[:, keep], nn[:, keep], wo[:, keep]
    q = {"x": x, "n": nn, "wo": wo, "albedo": rng.uniform(0.3, 1.0, (c, x.shape[1]))}
    assert x.shape[1] >= 12
    G = rng.standard_normal((c, x.shape[1]))
    an = oracle.hybrid_bwd(f["mean"], f["quat"], f["logscale"], f["spectrum"], x, nn, wo, G,
                           albedo=q["albedo"], **kw)
    for key in ("mean", "quat", "logscale", "spectrum"):
        num = np.zeros_like(f[key])
        for idx in np.ndindex(*f[key].shape):
            fp = {k: v.copy() for k, v in f.items()}
            fm = {k: v.copy() for k, v in f.items()}
            fp[key][idx] += 1e-6
            fm[key][idx] -= 1e-6
            num[idx] = (_hybrid_objective(fp, q, G, kw) - _hybrid_objective(fm, q, G, kw)) / 2e-6
        err = np.linalg.norm(num - an[key]) / max(np.linalg.norm(an[key]), 1e-300)
        assert err < 1e-6, (key, err)
        assert np.linalg.norm(an[key]) > 0.0


def test_hybrid_gradient_with_a_ball_holding_everything_is_the_untruncated_gradient():
    fnp, qnp = synth.config1_random(seed=34, n=40, m=30, albedo=True)
    G = np.random.default_rng(34).standard_normal((3, 30))
    for mode in (oracle.GPF_SUM, oracle.GPF_NORMALIZED):
        a = oracle.hybrid_bwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, qnp.x, qnp.n,
                              qnp.wo, G, qnp.albedo, mode=mode, r_max=0.05, ball_r=10.0, k_min=3)
        b = oracle.radiance_bwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, qnp.x, qnp.n,
                                qnp.wo, G, qnp.albedo, mode=mode, r_max=0.05,
                                cutoff_sigma=math.inf)
        for k in ("mean", "quat", "logscale", "spectrum"):
            np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-14 * np.abs(b[k]).max())


def test_hybrid_gradient_of_a_knn_only_selection_on_a_line():
    """kNN only (k_min = 2) at the origin of the line field: only the two
    nearest Gaussians get gradients; d O / d Phi_i = w_i for them (GPF_SUM),
    and the others are exactly zero."""
    dists = [0.01, 0.05, -0.09, 0.2]
    mean, quat, lsc, spec = _line_field(dists, [1.0, 2.0, 4.0, 8.0])
    x = np.zeros((3, 1))
    nrm = np.array([[0.0], [0.0], [1.0]])
    g = oracle.hybrid_bwd(mean, quat, lsc, spec, x, nrm, nrm, np.ones((1, 1)),
                          mode=oracle.GPF_SUM, r_max=0.02, ball_r=0.0, k_min=2)
    np.testing.assert_allclose(g["spectrum"][0], [_w_line(0.01), _w_line(0.05), 0.0, 0.0],
                               rtol=1e-13, atol=0)
    assert np.all(g["mean"][:, 2:] == 0) and np.all(g["logscale"][:, 2:] == 0)
