"""Shared helpers of the GPU tests: run the CUDA path through the binding,
run the oracle on the same seeded inputs, and measure the error."""

import math

import numpy as np

import oracle

FWD_TOL = 1e-5      # relative radiance error (scale: rho * sum_i w_i |Phi_i|)
# float32 evaluates w = exp(E), E = -Q/2 - 3 t^2, so w carries the absolute
# error of E as a relative error. The Mahalanobis part contributes a few
# u |Q/2| (u = 2^-24). The falloff part depends on the float32 distance d
# (relative error <= 2u after the sum of squares and the square root), with
# t = (d - r)/r: |d(3 t^2)| = 6 t (d/r) 2u = 12 u t (t + 1), which is at most
# 8 u * 3 t^2 for t >= 1 (and below 24 u, under FWD_TOL, for t < 1). So the
# error of E is at most 8 u |E|, and where the largest E at a hit point is
# far below zero that exceeds FWD_TOL: the tolerance there is
# EXP_COND * u * |E_max|.
U32 = 2.0 ** -24
EXP_COND = 8.0
GRAD_TOL = 1e-4     # normwise relative error per gradient tensor
DENOM_FLOOR = 1e-20


def gpu_fwd(gpf, fnp, qnp, mode, r_max, cutoff, cell=0.1, brute=False, idx=None):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    field = gpf.Field.from_numpy(fnp)
    queries = gpf.Queries.from_numpy(qnp)
    if idx is None:
        idx = make_index(field, queries, query_cell=cell, cutoff_sigma=cutoff, brute_force=brute)
    idx.build(field, queries)
    out, z = gpf.gpf_radiance_fwd(idx, field, queries, mode, r_max=r_max)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), z.cpu().numpy().astype(np.float64), idx, \
        (field, queries, out, z)


def oracle_fwd(fnp, qnp, mode, r_max, cutoff, sel=None):
    x, n, wo = qnp.x, qnp.n, qnp.wo
    alb, val = qnp.albedo, qnp.valid
    if sel is not None:
        x, n, wo = x[:, sel], n[:, sel], wo[:, sel]
        alb = None if alb is None else alb[:, sel]
        val = None if val is None else val[sel]
    return oracle.radiance_fwd(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum, x, n, wo, alb, val,
                               mode=mode, r_max=r_max, cutoff_sigma=cutoff)


# |E_max| above which the relaxed bar EXP_COND * u * |E_max| exceeds FWD_TOL
# (about 21: every weight at the hit point below e^-21).
RELAXED_FROM = FWD_TOL / (EXP_COND * U32)
# (test, points compared, points under the relaxed bar, largest error of
# those relative to FWD_TOL) of every forward comparison, reported at the end
# of the session.
RELAXED_LOG = []


def fwd_rel_err(out, ref, keep=None):
    """max over kept points of |O - O_ref| / max(rho sum w |Phi|, floor),
    divided by that point's tolerance relative to FWD_TOL (so the result is
    compared with FWD_TOL). Logs how many compared points were judged under
    the relaxed bar (RELAXED_LOG)."""
    import os
    err = np.abs(out - ref["out"]) / np.maximum(ref["denom"], DENOM_FLOOR)
    e_abs = np.abs(np.nan_to_num(ref["logw_max"], neginf=0.0))
    tol = np.maximum(FWD_TOL, EXP_COND * U32 * e_abs)
    err = err * (FWD_TOL / tol)[None, :]
    if keep is None:
        keep = ~ref["near_cutoff"]
    zero_ok = np.all(out[:, ref["denom"].max(axis=0) == 0] == 0)
    relaxed = keep & (e_abs > RELAXED_FROM) & (ref["denom"].max(axis=0) > 0)
    raw = np.abs(out - ref["out"]) / np.maximum(ref["denom"], DENOM_FLOOR)
    RELAXED_LOG.append((os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0],
                        int(keep.sum()), int(relaxed.sum()),
                        float(raw[:, relaxed].max() / FWD_TOL) if relaxed.any() else 0.0))
    return float(err[:, keep].max()) if keep.any() else 0.0, zero_ok


def grad_err(a, b):
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def sample_active(qnp, k, seed=0, tail=32):
    """k random active hit points plus the last `tail` indices (the ragged end)."""
    m = qnp.m
    act = np.flatnonzero((qnp.valid if qnp.valid is not None else np.ones(m, bool)).astype(bool)
                         & (np.sum(qnp.n.astype(np.float64) * qnp.wo, axis=0) > 0))
    rng = np.random.default_rng(seed)
    pick = rng.choice(act, size=min(k, act.size), replace=False) if act.size else act
    return np.unique(np.concatenate([pick, np.arange(max(0, m - tail), m)]))


INF = math.inf
