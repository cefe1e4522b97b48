"""FP64 brute-force oracle: radiance, gradient, MSE, Adam.

TEST INFRASTRUCTURE ONLY (see the package docstring). Plain float64 numpy,
a loop over chunks of queries, every Gaussian visited for every query; no
spatial index, no fusion, no reordering beyond what the definitions state.

Notation follows the paper: Gaussian i has mean mu_i, rotation q_i (unit
quaternion, stored (w, x, y, z) and normalised here), scale s_i = exp(l_i)
and spectral flux Phi_i in R^C; Sigma_i = R S S^T R^T and the precision is
Lambda_i = R S^-2 R^T (Sec. 4.1). For a hit point x with normal n, direction
to the viewer w_o and albedo rho:

    d   = x - mu_i
    u   = S^-1 R^T d          (local frame, per-axis divided by the scale)
    Q   = u . u = d^T Lambda_i d
    psi = 1 if |d| <= r else exp(-3 t^2), t = (|d| - r) / max(r, 1e-6)
    w_i = exp(-Q / 2) psi      (Sec. 4.2, aggregation equation)
    L   = sum_i w_i Phi_i,  Z = sum_i w_i
    O   = rho * L * [n.w_o > 0]                    (mode SUM)
    O   = rho * L / max(Z, eps) * [n.w_o > 0]      (mode NORMALIZED)

The neighbourhood is every Gaussian with Q <= cutoff^2 (cutoff = 3, the 3-sigma
ellipsoid), or every Gaussian when cutoff is infinite (brute force).
"""

from __future__ import annotations

import math
from typing import Dict, Optional

import numpy as np

GPF_SUM = 0
GPF_NORMALIZED = 1

_F64 = np.float64


def quat_to_rotmat(qhat: np.ndarray) -> np.ndarray:
    """Rotation matrix of unit quaternions (w, x, y, z), shape [..., 4] -> [..., 3, 3].

    Textbook form: column j of R is the j-th local axis expressed in world
    coordinates (Sec. 4.1: the rotation is a unit quaternion)."""
    w, x, y, z = (qhat[..., 0], qhat[..., 1], qhat[..., 2], qhat[..., 3])
    R = np.empty(qhat.shape[:-1] + (3, 3), dtype=_F64)
    R[..., 0, 0] = 1.0 - 2.0 * (y * y + z * z)
    R[..., 0, 1] = 2.0 * (x * y - w * z)
    R[..., 0, 2] = 2.0 * (x * z + w * y)
    R[..., 1, 0] = 2.0 * (x * y + w * z)
    R[..., 1, 1] = 1.0 - 2.0 * (x * x + z * z)
    R[..., 1, 2] = 2.0 * (y * z - w * x)
    R[..., 2, 0] = 2.0 * (x * z - w * y)
    R[..., 2, 1] = 2.0 * (y * z + w * x)
    R[..., 2, 2] = 1.0 - 2.0 * (x * x + y * y)
    return R


def _rotmat_partials(qhat: np.ndarray) -> np.ndarray:
    """dR/dq_a for a = w, x, y, z: shape [N, 4, 3, 3] (entrywise derivative of
    the textbook matrix above with respect to each quaternion component)."""
    w, x, y, z = (qhat[:, 0], qhat[:, 1], qhat[:, 2], qhat[:, 3])
    zero = np.zeros_like(w)
    P = np.empty((qhat.shape[0], 4, 3, 3), dtype=_F64)
    P[:, 0] = np.stack([np.stack([zero, -2 * z, 2 * y], -1),
                        np.stack([2 * z, zero, -2 * x], -1),
                        np.stack([-2 * y, 2 * x, zero], -1)], -2)
    P[:, 1] = np.stack([np.stack([zero, 2 * y, 2 * z], -1),
                        np.stack([2 * y, -4 * x, -2 * w], -1),
                        np.stack([2 * z, 2 * w, -4 * x], -1)], -2)
    P[:, 2] = np.stack([np.stack([-4 * y, 2 * x, 2 * w], -1),
                        np.stack([2 * x, zero, 2 * z], -1),
                        np.stack([-2 * w, 2 * z, -4 * y], -1)], -2)
    P[:, 3] = np.stack([np.stack([-4 * z, -2 * w, 2 * x], -1),
                        np.stack([2 * w, -4 * z, 2 * y], -1),
                        np.stack([2 * x, 2 * y, zero], -1)], -2)
    return P


def falloff_psi(dist: np.ndarray, r_max: float) -> np.ndarray:
    """Soft distance falloff psi(|d|) of Sec. 4.2, in the form the query listing of
    Algorithm S3 gives: 1 inside the radius r, exp(-3 t^2) outside with
    t = (|d| - r) / max(r, 1e-6). An infinite radius disables it (psi = 1)."""
    dist = np.asarray(dist, dtype=_F64)
    if not math.isfinite(r_max):
        return np.ones_like(dist)
    t = (dist - r_max) / max(r_max, 1e-6)
    return np.where(dist <= r_max, 1.0, np.exp(-3.0 * t * t))


def _falloff_dpsi_ddist(dist: np.ndarray, r_max: float) -> np.ndarray:
    """d psi / d |d|: 0 inside r, -6 t / max(r, 1e-6) * psi outside."""
    if not math.isfinite(r_max):
        return np.zeros_like(dist)
    rr = max(r_max, 1e-6)
    t = (dist - r_max) / rr
    return np.where(dist <= r_max, 0.0, -6.0 * t / rr * np.exp(-3.0 * t * t))


class _Prepared:
    """Per-Gaussian quantities in float64: mu [N,3], qhat [N,4], |q| [N],
    R [N,3,3], s [N,3], Phi [N,C]."""

    def __init__(self, mean, quat, logscale, spectrum):
        self.mu = np.asarray(mean, dtype=_F64).T.copy()
        q = np.asarray(quat, dtype=_F64).T
        self.qnorm = np.linalg.norm(q, axis=1)
        self.qhat = q / self.qnorm[:, None]
        self.R = quat_to_rotmat(self.qhat)
        self.s = np.exp(np.asarray(logscale, dtype=_F64).T)
        self.phi = np.asarray(spectrum, dtype=_F64).T.copy()
        self.n = self.mu.shape[0]
        self.c = self.phi.shape[1]


def _pairs(P: _Prepared, xs: np.ndarray, r_max: float, cutoff_sigma: float):
    """All (query, Gaussian) pair terms for a chunk of queries xs [m,3]:
    d [m,N,3], u [m,N,3], Q [m,N], dist [m,N], included [m,N] (bool), w [m,N]."""
    d = xs[:, None, :] - P.mu[None, :, :]
    # u_j = (R^T d)_j / s_j = sum_k R_kj d_k / s_j
    u = np.empty_like(d)
    for j in range(3):
        u[..., j] = (d[..., 0] * P.R[None, :, 0, j] + d[..., 1] * P.R[None, :, 1, j]
                     + d[..., 2] * P.R[None, :, 2, j]) / P.s[None, :, j]
    Q = u[..., 0] ** 2 + u[..., 1] ** 2 + u[..., 2] ** 2
    if math.isfinite(cutoff_sigma):
        inc = Q <= cutoff_sigma * cutoff_sigma
    else:
        inc = np.ones(Q.shape, dtype=bool)
    dist = np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2 + d[..., 2] ** 2)
    w = np.where(inc, np.exp(-0.5 * Q) * falloff_psi(dist, r_max), 0.0)
    return d, u, Q, dist, inc, w


def _chunk(n_gauss: int) -> int:
    return max(1, (1 << 21) // max(n_gauss, 1))


def _query_mask(n, wo, valid, m):
    nd = np.sum(np.asarray(n, dtype=_F64) * np.asarray(wo, dtype=_F64), axis=0)
    mask = nd > 0.0
    if valid is not None:
        mask &= np.asarray(valid).astype(bool)
    return mask


def radiance_fwd(mean, quat, logscale, spectrum, x, n, wo, albedo=None, valid=None,
                 mode: int = GPF_SUM, r_max: float = math.inf, eps: float = 1e-6,
                 cutoff_sigma: float = 3.0, band: float = 1e-4) -> Dict[str, np.ndarray]:
    """Forward radiance at M hit points (arrays in the C library's SoA layout).

    Returns out [C,M] (the output O), L [C,M] (sum_i w_i Phi_i), Z [M]
    (sum_i w_i), n_pairs [M] (included pairs), denom [C,M] (rho * sum_i w_i
    |Phi_i|, the scale of the relative error), near_cutoff [M] (True when some
    pair has |Q - cutoff^2| < band, where float32 and float64 may classify the
    pair differently), mask [M] (valid and n.w_o > 0) and logw_max [M] (log of
    the largest weight, -inf if none)."""
    P = _Prepared(mean, quat, logscale, spectrum)
    X = np.asarray(x, dtype=_F64).T
    M, C = X.shape[0], P.c
    L = np.zeros((M, C))
    Lab = np.zeros((M, C))
    Z = np.zeros(M)
    npairs = np.zeros(M, dtype=np.int64)
    near = np.zeros(M, dtype=bool)
    logw_max = np.full(M, -np.inf)
    cut2 = cutoff_sigma * cutoff_sigma
    step = _chunk(P.n)
    for a in range(0, M, step):
        b = min(M, a + step)
        _, _, Q, _, inc, w = _pairs(P, X[a:b], r_max, cutoff_sigma)
        L[a:b] = w @ P.phi
        Lab[a:b] = w @ np.abs(P.phi)
        Z[a:b] = w.sum(axis=1)
        npairs[a:b] = inc.sum(axis=1)
        with np.errstate(divide="ignore"):
            logw_max[a:b] = np.log(w.max(axis=1)) if P.n else -np.inf
        if math.isfinite(cutoff_sigma):
            near[a:b] = np.any(np.abs(Q - cut2) < band, axis=1)
    mask = _query_mask(n, wo, valid, M)
    rho = np.ones((M, C)) if albedo is None else np.asarray(albedo, dtype=_F64).T
    if mode == GPF_SUM:
        out = rho * L
    elif mode == GPF_NORMALIZED:
        out = rho * L / np.maximum(Z, eps)[:, None]
    else:
        raise ValueError("mode must be GPF_SUM or GPF_NORMALIZED")
    out = np.where(mask[:, None], out, 0.0)
    denom = rho * Lab
    if mode == GPF_NORMALIZED:
        denom = denom / np.maximum(Z, eps)[:, None]
    denom = np.where(mask[:, None], denom, 0.0)
    return {"out": out.T.copy(), "L": L.T.copy(), "Z": Z, "n_pairs": npairs,
            "denom": denom.T.copy(), "near_cutoff": near, "mask": mask, "logw_max": logw_max}


def radiance_bwd(mean, quat, logscale, spectrum, x, n, wo, grad_out, albedo=None,
                 valid=None, mode: int = GPF_SUM, r_max: float = math.inf,
                 eps: float = 1e-6, cutoff_sigma: float = 3.0) -> Dict[str, np.ndarray]:
    """Gradient of sum_{c,m} grad_out[c,m] * O[c,m] with respect to the raw
    parameters: mean [3,N], quat [4,N] (raw, through the normalisation),
    logscale [3,N], spectrum [C,N]. Chain rule through each step of the
    forward (Sec. 4.2, Differentiable Accumulation); the indicator Q <= cutoff^2
    is piecewise constant and contributes no derivative."""
    P = _Prepared(mean, quat, logscale, spectrum)
    X = np.asarray(x, dtype=_F64).T
    M, C, N = X.shape[0], P.c, P.n
    G = np.asarray(grad_out, dtype=_F64).T
    fwd = radiance_fwd(mean, quat, logscale, spectrum, x, n, wo, albedo, valid, mode,
                       r_max, eps, cutoff_sigma)
    mask = fwd["mask"]
    rho = np.ones((M, C)) if albedo is None else np.asarray(albedo, dtype=_F64).T
    gamma = G * rho * mask[:, None]          # d loss / d (L or L/max(Z,eps))
    L, Z = fwd["L"].T, fwd["Z"]
    if mode == GPF_SUM:
        dL = gamma                            # d loss / d L_c
        dZ = np.zeros(M)                      # d loss / d Z
    else:
        big = Z > eps
        Zc = np.where(big, Z, eps)
        dL = gamma / Zc[:, None]
        dZ = np.where(big, -np.sum(gamma * L, axis=1) / (Zc * Zc), 0.0)

    g_mu = np.zeros((N, 3))
    g_R = np.zeros((N, 3, 3))
    g_l = np.zeros((N, 3))
    g_phi = np.zeros((N, C))
    step = _chunk(N)
    for a in range(0, M, step):
        b = min(M, a + step)
        d, u, Q, dist, inc, w = _pairs(P, X[a:b], r_max, cutoff_sigma)
        # d loss / d w_i for every pair: sum_c dL_c Phi_ic + dZ
        beta = dL[a:b] @ P.phi.T + dZ[a:b, None]
        bw = beta * w
        # d loss / d Phi_ic = sum_m dL_mc w_mi
        g_phi += w.T @ dL[a:b]
        # dw/dl_j = w u_j^2
        g_l += np.einsum("mn,mnj->nj", bw, u * u)
        # dw/dR_kj = -w u_j d_k / s_j
        g_R -= np.einsum("mn,mnk,mnj->nkj", bw, d, u) / P.s[:, None, :]
        # dw/dmu_k through the Gaussian factor: w sum_j u_j R_kj / s_j
        g_mu += np.einsum("mn,mnj,nkj->nk", bw, u, P.R / P.s[:, None, :])
        # dw/dmu_k through psi: -g psi'(|d|) d_k / |d|
        dpsi = _falloff_dpsi_ddist(dist, r_max)
        with np.errstate(divide="ignore", invalid="ignore"):
            coef = np.where(inc & (dist > 0.0),
                            -beta * np.exp(-0.5 * Q) * dpsi / np.where(dist > 0, dist, 1.0),
                            0.0)
        g_mu += np.einsum("mn,mnk->nk", coef, d)
    # R = R(qhat): d loss / d qhat_a = sum_kj g_R_kj dR_kj/dqhat_a
    g_qhat = np.einsum("nkj,nakj->na", g_R, _rotmat_partials(P.qhat))
    # qhat = q / |q|: d qhat / d q = (I - qhat qhat^T) / |q|
    g_q = (g_qhat - P.qhat * np.sum(P.qhat * g_qhat, axis=1, keepdims=True)) / P.qnorm[:, None]
    return {"mean": g_mu.T.copy(), "quat": g_q.T.copy(), "logscale": g_l.T.copy(),
            "spectrum": g_phi.T.copy(), "fwd": fwd}


def hybrid_fwd(mean, quat, logscale, spectrum, x, n, wo, albedo=None, valid=None,
               mode: int = GPF_NORMALIZED, r_max: float = 0.02, eps: float = 1e-6,
               ball_r: float = 0.02, k_min: int = 3, band: float = 1e-5) -> Dict[str, np.ndarray]:
    """The paper's hybrid neighbourhood (Sec. 4.2, Neighborhood Search; the
    query listing of Algorithm S3): N(x) = the Gaussians whose mean lies
    within ball_r of x if there are at least k_min of them, else the k_min
    nearest means (ties: the smaller index); the union with the ball is the
    same set, since every mean in the ball is nearer than every mean outside.
    Weights w_i = exp(-Q_i/2) psi(|d_i|) over N(x), no truncation; output as
    radiance_fwd (GPF_SUM or GPF_NORMALIZED).

    Returns out, L, Z, denom (as radiance_fwd), logw_max [M] (the largest log
    weight in N(x)), n_nb [M] (|N(x)|), knn [M] (the k_min nearest were used)
    and near [M]: the selection is sensitive to rounding (a mean within
    band*ball_r^2 of the ball's edge in squared distance, or, in kNN mode, the
    k-th and (k+1)-th squared distances within a relative band of each other)."""
    P = _Prepared(mean, quat, logscale, spectrum)
    X = np.asarray(x, dtype=_F64).T
    M, C, N = X.shape[0], P.c, P.n
    mask = _query_mask(n, wo, valid, M)
    rho = np.ones((M, C)) if albedo is None else np.asarray(albedo, dtype=_F64).T
    L = np.zeros((M, C))
    Z = np.zeros(M)
    den = np.zeros((M, C))
    n_nb = np.zeros(M, dtype=np.int64)
    knn = np.zeros(M, dtype=bool)
    near = np.zeros(M, dtype=bool)
    logw = np.full(M, -np.inf)
    r2 = float(ball_r) ** 2
    idx = np.arange(N)
    step = _chunk(N)
    for a in range(0, M, step):
        xs = X[a:a + step]
        d, _, _, _, _, w = _pairs(P, xs, r_max, math.inf)        # every pair, untruncated
        d2 = d[..., 0] ** 2 + d[..., 1] ** 2 + d[..., 2] ** 2
        for j in range(xs.shape[0]):
            ball = d2[j] <= r2
            sel = ball
            if ball.sum() < k_min:
                order = np.lexsort((idx, d2[j]))                 # by distance, then index
                sel = np.zeros(N, dtype=bool)
                sel[order[:min(k_min, N)]] = True
                knn[a + j] = True
                if N > k_min:
                    dk, dk1 = d2[j][order[k_min - 1]], d2[j][order[k_min]]
                    near[a + j] |= abs(dk1 - dk) <= band * max(dk, 1e-300)
            if r2 > 0:
                near[a + j] |= bool(np.any(np.abs(d2[j] - r2) <= band * r2))
            wj = np.where(sel, w[j], 0.0)
            with np.errstate(divide="ignore"):
                logw[a + j] = np.log(wj.max()) if sel.any() else -np.inf
            L[a + j] = wj @ P.phi
            Z[a + j] = wj.sum()
            den[a + j] = wj @ np.abs(P.phi)
            n_nb[a + j] = sel.sum()
    g = mask.astype(_F64)[:, None]
    if mode == GPF_NORMALIZED:
        zz = np.maximum(Z, eps)[:, None]
        out, denom = rho * L / zz * g, rho * den / zz * g
    else:
        out, denom = rho * L * g, rho * den * g
    return {"out": out.T, "L": L.T, "Z": Z * mask, "denom": denom.T, "n_nb": n_nb * mask,
            "knn": knn & mask, "near": near & mask, "logw_max": logw}


def hybrid_bwd(mean, quat, logscale, spectrum, x, n, wo, grad_out, albedo=None, valid=None,
               mode: int = GPF_NORMALIZED, r_max: float = 0.02, eps: float = 1e-6,
               ball_r: float = 0.02, k_min: int = 3) -> Dict[str, np.ndarray]:
    """Gradient of sum_{c,m} grad_out[c,m] * O[c,m] for the hybrid
    neighbourhood of hybrid_fwd (Sec. 4.2, Neighborhood Search and
    Differentiable Accumulation): the selection N(x) (the ball of radius
    ball_r around x, or the k_min nearest means when the ball holds fewer) is
    piecewise constant in the parameters and contributes no derivative; over
    the selected pairs the chain rule is the one of radiance_bwd with the
    untruncated weights w_i = exp(-Q_i/2) psi(|d_i|). Returns mean, quat, logscale,
    spectrum (as radiance_bwd) and fwd (hybrid_fwd's result)."""
    P = _Prepared(mean, quat, logscale, spectrum)
    X = np.asarray(x, dtype=_F64).T
    M, C, N = X.shape[0], P.c, P.n
    G = np.asarray(grad_out, dtype=_F64).T
    fwd = hybrid_fwd(mean, quat, logscale, spectrum, x, n, wo, albedo, valid, mode, r_max, eps,
                     ball_r, k_min)
    mask = _query_mask(n, wo, valid, M)
    rho = np.ones((M, C)) if albedo is None else np.asarray(albedo, dtype=_F64).T
    gamma = G * rho * mask[:, None]
    L, Z = fwd["L"].T, fwd["Z"]
    if mode == GPF_SUM:
        dL, dZ = gamma, np.zeros(M)
    else:
        big = Z > eps
        Zc = np.where(big, Z, eps)
        dL = gamma / Zc[:, None]
        dZ = np.where(big, -np.sum(gamma * L, axis=1) / (Zc * Zc), 0.0)
    g_mu = np.zeros((N, 3))
    g_R = np.zeros((N, 3, 3))
    g_l = np.zeros((N, 3))
    g_phi = np.zeros((N, C))
    r2 = float(ball_r) ** 2
    idx = np.arange(N)
    step = _chunk(N)
    for a in range(0, M, step):
        b = min(M, a + step)
        d, u, Q, dist, _, w_all = _pairs(P, X[a:b], r_max, math.inf)
        d2 = d[..., 0] ** 2 + d[..., 1] ** 2 + d[..., 2] ** 2
        # the selection of hybrid_fwd, point by point
        sel = np.zeros((b - a, N), dtype=bool)
        for j in range(b - a):
            ball = d2[j] <= r2
            if ball.sum() >= k_min:
                sel[j] = ball
            else:
                order = np.lexsort((idx, d2[j]))
                sel[j, order[:min(k_min, N)]] = True
        w = np.where(sel, w_all, 0.0)
        beta = dL[a:b] @ P.phi.T + dZ[a:b, None]
        bw = beta * w
        g_phi += w.T @ dL[a:b]
        g_l += np.einsum("mn,mnj->nj", bw, u * u)
        g_R -= np.einsum("mn,mnk,mnj->nkj", bw, d, u) / P.s[:, None, :]
        g_mu += np.einsum("mn,mnj,nkj->nk", bw, u, P.R / P.s[:, None, :])
        dpsi = _falloff_dpsi_ddist(dist, r_max)
        with np.errstate(divide="ignore", invalid="ignore"):
            coef = np.where(sel & (dist > 0.0),
                            -beta * np.exp(-0.5 * Q) * dpsi / np.where(dist > 0, dist, 1.0),
                            0.0)
        g_mu += np.einsum("mn,mnk->nk", coef, d)
    g_qhat = np.einsum("nkj,nakj->na", g_R, _rotmat_partials(P.qhat))
    g_q = (g_qhat - P.qhat * np.sum(P.qhat * g_qhat, axis=1, keepdims=True)) / P.qnorm[:, None]
    return {"mean": g_mu.T.copy(), "quat": g_q.T.copy(), "logscale": g_l.T.copy(),
            "spectrum": g_phi.T.copy(), "fwd": fwd}


def disk_kde(position, flux, x, n, wo, radius: float, albedo=None, valid=None,
             band: float = 1e-5) -> Dict[str, np.ndarray]:
    """The per-view photon density estimate that the field replaces (Sec. 3.2,
    Eq. kde; the gather of Algorithm S1): at hit point x, the flux of every
    photon p with |x - x_p| <= r, divided by the disk area pi r^2, modulated
    like the field's query (albedo times the hemisphere gate):

        O_c = rho_c (1 / (pi r^2)) sum_{p : |x - x_p| <= r} Phi_pc [n.w_o > 0]

    position [3,P], flux [C,P]. Returns out [C,M], count [M] (photons
    gathered), denom [C,M] (the same sum of |Phi|, the scale of the error),
    near [M] (some photon lies within band r^2 of the disk's edge in squared
    distance, where float32 and float64 may disagree)."""
    pos = np.asarray(position, dtype=_F64).T
    phi = np.asarray(flux, dtype=_F64).T
    X = np.asarray(x, dtype=_F64).T
    M, C = X.shape[0], phi.shape[1]
    r2 = float(radius) ** 2
    mask = _query_mask(n, wo, valid, M)
    rho = np.ones((M, C)) if albedo is None else np.asarray(albedo, dtype=_F64).T
    out = np.zeros((M, C))
    den = np.zeros((M, C))
    count = np.zeros(M)
    near = np.zeros(M, dtype=bool)
    step = _chunk(pos.shape[0])
    for a in range(0, M, step):
        xs = X[a:a + step]
        d2 = np.sum((xs[:, None, :] - pos[None, :, :]) ** 2, axis=2)
        inc = d2 <= r2
        out[a:a + step] = inc.astype(_F64) @ phi
        den[a:a + step] = inc.astype(_F64) @ np.abs(phi)
        count[a:a + step] = inc.sum(axis=1)
        near[a:a + step] = np.any(np.abs(d2 - r2) <= band * r2, axis=1)
    area = np.pi * r2
    g = mask[:, None].astype(_F64)
    return {"out": (rho * out / area * g).T, "denom": (rho * den / area * g).T,
            "count": count * mask, "near": near}


def mse_loss(out, target, valid=None) -> float:
    """Sec. 4.3: (1/|V|) sum_{x in V} |O(x) - O_ref(x)|_2^2 over the valid points."""
    O = np.asarray(out, dtype=_F64)
    T = np.asarray(target, dtype=_F64)
    v = np.ones(O.shape[1], dtype=bool) if valid is None else np.asarray(valid).astype(bool)
    nv = int(v.sum())
    if nv == 0:
        return 0.0
    return float(np.sum((O[:, v] - T[:, v]) ** 2) / nv)


def mse_loss_grad(out, target, valid=None) -> np.ndarray:
    """d mse_loss / d out = 2 (O - O_ref) / |V| on valid points, 0 elsewhere."""
    O = np.asarray(out, dtype=_F64)
    T = np.asarray(target, dtype=_F64)
    v = np.ones(O.shape[1], dtype=bool) if valid is None else np.asarray(valid).astype(bool)
    nv = int(v.sum())
    g = np.zeros_like(O)
    if nv:
        g[:, v] = 2.0 * (O[:, v] - T[:, v]) / nv
    return g


def adam_step(param, grad, m, v, step: int, lr: float = 5e-4, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba, bias-corrected; the optimiser of Sec. A.2
    with its learning rate 5e-4). `step` is the 1-based index of this update.
    Returns (param, m, v) as new float64 arrays."""
    p = np.asarray(param, dtype=_F64)
    g = np.asarray(grad, dtype=_F64)
    m1 = beta1 * np.asarray(m, dtype=_F64) + (1.0 - beta1) * g
    v1 = beta2 * np.asarray(v, dtype=_F64) + (1.0 - beta2) * g * g
    mhat = m1 / (1.0 - beta1 ** step)
    vhat = v1 / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m1, v1
