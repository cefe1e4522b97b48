"""Seeded generators: random fields, caustic-like photon maps, pinhole hit points.

Every generator takes an integer seed and draws from numpy's PCG64, so a
(seed, size) pair always yields the same bytes. Arrays are structure-of-arrays
float32 (one row per component), which is the layout the C library takes.

The analytic scene stands in for the paper's Mitsuba scenes (Sec. 5.1), which
are not available: a floor z = 0 on [-4, 4]^2 and a unit sphere centred at
(0, 0, 1). Photons are deposited 70 % in a mixture of eight anisotropic 2D
Gaussians on the floor (a caustic-like pattern) and 30 % uniformly by area over
floor and sphere. One Gaussian per photon follows the paper's initialisation
(Sec. 4.1: mean at the photon, flux from the photon, random rotation), with the
isotropic scale taken from the distance to the 8th nearest photon.
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

FLOOR_HALF = 4.0
SPHERE_CENTRE = np.array([0.0, 0.0, 1.0])
SPHERE_RADIUS = 1.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


@dataclasses.dataclass
class Field:
    """N Gaussians: mean [3,N], quat [4,N] (w,x,y,z, not necessarily unit),
    logscale [3,N] (scale = exp(logscale)), spectrum [C,N]; all float32."""

    mean: np.ndarray
    quat: np.ndarray
    logscale: np.ndarray
    spectrum: np.ndarray

    @property
    def n(self) -> int:
        return int(self.mean.shape[1])

    @property
    def channels(self) -> int:
        return int(self.spectrum.shape[0])

    def copy(self) -> "Field":
        return Field(self.mean.copy(), self.quat.copy(), self.logscale.copy(),
                     self.spectrum.copy())


@dataclasses.dataclass
class Queries:
    """M hit points: x, n (unit normal), wo (unit, towards the viewer), all
    [3,M] float32; albedo [C,M] float32 or None (= 1); valid [M] uint8 or
    None (= all valid). view_offsets [V+1] int64 and view_shapes [(H, W)]
    describe how the queries split into row-major views."""

    x: np.ndarray
    n: np.ndarray
    wo: np.ndarray
    albedo: Optional[np.ndarray] = None
    valid: Optional[np.ndarray] = None
    view_offsets: Optional[np.ndarray] = None
    view_shapes: Optional[List[tuple]] = None

    @property
    def m(self) -> int:
        return int(self.x.shape[1])


def _unit_rows(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=0, keepdims=True)


def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform rotations: a normalised standard-normal 4-vector per Gaussian."""
    q = rng.standard_normal((4, n))
    return q / np.linalg.norm(q, axis=0, keepdims=True)


def config1_random(seed: int = 0, n: int = 4096, m: int = 16384, channels: int = 3,
                   albedo: bool = False) -> tuple:
    """Unit-cube field and queries: means U[0,1]^3, log-scales N(-3, 0.5) per
    axis, uniform unit quaternions, spectrum U[0,1]^C; hit points U[0,1]^3
    with uniformly random unit normals and view directions."""
    rng = _rng(seed)
    field = Field(
        mean=_f32(rng.uniform(0.0, 1.0, (3, n))),
        quat=_f32(random_quaternions(rng, n)),
        logscale=_f32(rng.normal(-3.0, 0.5, (3, n))),
        spectrum=_f32(rng.uniform(0.0, 1.0, (channels, n))),
    )
    q = Queries(
        x=_f32(rng.uniform(0.0, 1.0, (3, m))),
        n=_f32(_unit_rows(rng.standard_normal((3, m)))),
        wo=_f32(_unit_rows(rng.standard_normal((3, m)))),
    )
    if albedo:
        q.albedo = _f32(rng.uniform(0.2, 1.0, (channels, m)))
    q.valid = np.ones(m, dtype=np.uint8)
    q.view_offsets = np.array([0, m], dtype=np.int64)
    return field, q


def caustic_photons(n_photons: int, seed: int = 0, channels: int = 3,
                    blob_fraction: float = 0.7, n_blobs: int = 8) -> tuple:
    """Photon positions [n,3] float64 and fluxes [n,C] float64.

    blob_fraction of the photons come from an equal-weight mixture of n_blobs
    anisotropic 2D Gaussians on the floor (centres U[-2.5,2.5]^2, two principal
    standard deviations log-uniform in [0.02, 0.3], orientation U[0, pi));
    the rest are uniform by area over the floor and the sphere. Fluxes are
    Exp(1) per channel. The photon order is shuffled, as in a traced map."""
    rng = _rng(seed)
    n_blob = int(round(blob_fraction * n_photons))
    n_unif = n_photons - n_blob

    centres = rng.uniform(-2.5, 2.5, (n_blobs, 2))
    stds = np.exp(rng.uniform(np.log(0.02), np.log(0.3), (n_blobs, 2)))
    angles = rng.uniform(0.0, np.pi, n_blobs)
    which = rng.integers(0, n_blobs, n_blob)
    z = rng.standard_normal((n_blob, 2)) * stds[which]
    c, s = np.cos(angles[which]), np.sin(angles[which])
    blob_xy = centres[which] + np.stack([c * z[:, 0] - s * z[:, 1],
                                         s * z[:, 0] + c * z[:, 1]], axis=1)
    # resample the rare points that fall off the floor
    for _ in range(64):
        bad = np.any(np.abs(blob_xy) > FLOOR_HALF, axis=1)
        if not bad.any():
            break
        blob_xy[bad] = rng.uniform(-FLOOR_HALF, FLOOR_HALF, (int(bad.sum()), 2))
    blob = np.concatenate([blob_xy, np.zeros((n_blob, 1))], axis=1)

    area_floor = (2 * FLOOR_HALF) ** 2
    area_sphere = 4.0 * np.pi * SPHERE_RADIUS ** 2
    on_sphere = rng.uniform(0.0, 1.0, n_unif) < area_sphere / (area_floor + area_sphere)
    ns = int(on_sphere.sum())
    unif = np.empty((n_unif, 3))
    unif[~on_sphere, :2] = rng.uniform(-FLOOR_HALF, FLOOR_HALF, (n_unif - ns, 2))
    unif[~on_sphere, 2] = 0.0
    dirs = rng.standard_normal((ns, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    unif[on_sphere] = SPHERE_CENTRE + SPHERE_RADIUS * dirs

    pos = np.concatenate([blob, unif], axis=0)
    flux = rng.exponential(1.0, (n_photons, channels))
    perm = rng.permutation(n_photons)
    return pos[perm], flux[perm]


def knn_distance(pos: np.ndarray, k: int = 8) -> np.ndarray:
    """Distance from each point to its k-th nearest other point."""
    from scipy.spatial import cKDTree

    tree = cKDTree(pos)
    d, _ = tree.query(pos, k=k + 1, workers=-1)
    return d[:, k]


def field_from_photons(pos: np.ndarray, flux: np.ndarray, seed: int = 0,
                       knn: int = 8, min_scale: float = 1e-5) -> Field:
    """One Gaussian per photon: mean = position, spectrum = flux, isotropic
    scale = distance to the knn-th nearest photon, uniformly random rotation."""
    rng = _rng(seed + 7919)
    n = pos.shape[0]
    s = np.maximum(knn_distance(pos, knn), min_scale)
    return Field(
        mean=_f32(pos.T),
        quat=_f32(random_quaternions(rng, n)),
        logscale=_f32(np.tile(np.log(s), (3, 1))),
        spectrum=_f32(flux.T),
    )


def _morton_keys(pos: np.ndarray, bits: int = 21) -> np.ndarray:
    lo, hi = pos.min(axis=0), pos.max(axis=0)
    span = np.maximum(hi - lo, 1e-12)
    qv = np.clip(((pos - lo) / span * ((1 << bits) - 1)).astype(np.uint64), 0, (1 << bits) - 1)
    key = np.zeros(pos.shape[0], dtype=np.uint64)
    for b in range(bits):
        for a in range(3):
            key |= ((qv[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    return key


def merge_photon_pairs(pos: np.ndarray, flux: np.ndarray) -> tuple:
    """Halve a photon map by merging consecutive photons in Morton order:
    position = flux-weighted mean, flux = sum."""
    order = np.argsort(_morton_keys(pos), kind="stable")
    pos, flux = pos[order], flux[order]
    n2 = pos.shape[0] // 2
    a, b = slice(0, 2 * n2, 2), slice(1, 2 * n2, 2)
    wa = flux[a].sum(axis=1, keepdims=True)
    wb = flux[b].sum(axis=1, keepdims=True)
    wsum = np.maximum(wa + wb, 1e-30)
    mpos = (pos[a] * wa + pos[b] * wb) / wsum
    mflux = flux[a] + flux[b]
    if pos.shape[0] % 2:
        mpos = np.concatenate([mpos, pos[-1:]], axis=0)
        mflux = np.concatenate([mflux, flux[-1:]], axis=0)
    return mpos, mflux


def pinhole_hitpoints(eye: Sequence[float], look_at: Sequence[float], width: int,
                      height: int, vfov_deg: float = 45.0,
                      up: Sequence[float] = (0.0, 0.0, 1.0)) -> Queries:
    """First hits of the pixel-centre rays of a pinhole camera with the floor
    and the sphere. Pixels are row-major (row 0 at the top). Rays that miss
    both are marked invalid (x = 0, n = wo = +z)."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = np.asarray(look_at, dtype=np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, dtype=np.float64))
    right /= np.linalg.norm(right)
    cam_up = np.cross(right, fwd)
    tan_half = np.tan(np.radians(vfov_deg) / 2.0)
    aspect = width / height
    jj, ii = np.meshgrid(np.arange(width), np.arange(height))
    px = ((2.0 * (jj.ravel() + 0.5) / width) - 1.0) * tan_half * aspect
    py = (1.0 - (2.0 * (ii.ravel() + 0.5) / height)) * tan_half
    d = fwd[None, :] + px[:, None] * right[None, :] + py[:, None] * cam_up[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    m = d.shape[0]

    t_best = np.full(m, np.inf)
    nrm = np.zeros((m, 3))
    # floor z = 0 on [-4, 4]^2
    with np.errstate(divide="ignore", invalid="ignore"):
        tp = -eye[2] / d[:, 2]
    hp = eye[None, :] + tp[:, None] * d
    ok = (tp > 1e-6) & (np.abs(hp[:, 0]) <= FLOOR_HALF) & (np.abs(hp[:, 1]) <= FLOOR_HALF)
    t_best[ok] = tp[ok]
    nrm[ok] = np.array([0.0, 0.0, 1.0])
    # unit sphere
    oc = eye - SPHERE_CENTRE
    b = d @ oc
    cc = oc @ oc - SPHERE_RADIUS ** 2
    disc = b * b - cc
    hit = disc >= 0.0
    sq = np.sqrt(np.where(hit, disc, 0.0))
    ts = -b - sq
    ts = np.where(ts > 1e-6, ts, -b + sq)
    hit &= ts > 1e-6
    closer = hit & (ts < t_best)
    t_best[closer] = ts[closer]
    hs = eye[None, :] + ts[:, None] * d
    nrm[closer] = (hs[closer] - SPHERE_CENTRE) / SPHERE_RADIUS

    valid = np.isfinite(t_best)
    x = np.where(valid[:, None], eye[None, :] + np.where(valid, t_best, 0.0)[:, None] * d, 0.0)
    wo = np.where(valid[:, None], -d, np.array([0.0, 0.0, 1.0]))
    nrm = np.where(valid[:, None], nrm, np.array([0.0, 0.0, 1.0]))
    # on the floor the exact hit is z = 0; keep it exact after rounding
    return Queries(x=_f32(x.T), n=_f32(nrm.T), wo=_f32(wo.T), albedo=None,
                   valid=valid.astype(np.uint8),
                   view_offsets=np.array([0, m], dtype=np.int64),
                   view_shapes=[(height, width)])


def concat_queries(views: Sequence[Queries]) -> Queries:
    offs = np.zeros(len(views) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([v.m for v in views])
    alb = None
    if any(v.albedo is not None for v in views):
        c = next(v.albedo.shape[0] for v in views if v.albedo is not None)
        alb = _f32(np.concatenate([v.albedo if v.albedo is not None else
                                   np.ones((c, v.m), np.float32) for v in views], axis=1))
    return Queries(
        x=_f32(np.concatenate([v.x for v in views], axis=1)),
        n=_f32(np.concatenate([v.n for v in views], axis=1)),
        wo=_f32(np.concatenate([v.wo for v in views], axis=1)),
        albedo=alb,
        valid=np.concatenate([v.valid if v.valid is not None else np.ones(v.m, np.uint8)
                              for v in views]).astype(np.uint8),
        view_offsets=offs,
        view_shapes=[s for v in views for s in (v.view_shapes or [(1, v.m)])],
    )


def orbit_views(n_views: int = 8, width: int = 800, height: int = 800,
                radius: float = 6.0, cam_height: float = 3.0,
                look_at: Sequence[float] = (0.0, 0.0, 1.0),
                azimuth0_deg: float = 0.0) -> Queries:
    """n_views cameras evenly spaced in azimuth on a circle, all aimed at look_at."""
    views = []
    for k in range(n_views):
        a = np.radians(azimuth0_deg + 360.0 * k / n_views)
        eye = (radius * np.cos(a), radius * np.sin(a), cam_height)
        views.append(pinhole_hitpoints(eye, look_at, width, height))
    return concat_queries(views)


def uneven_views(n_views: int = 64, seed: int = 0,
                 sides: Sequence[int] = (256, 384, 512, 768, 1024)) -> Queries:
    """n_views square views of random side (uniform over `sides`), cameras at
    random azimuth, distance U[5,8] and height U[2,5], aimed at (0,0,0.5)."""
    rng = _rng(seed + 104729)
    views = []
    for _ in range(n_views):
        side = int(rng.choice(np.asarray(sides)))
        a = rng.uniform(0.0, 2.0 * np.pi)
        rad = rng.uniform(5.0, 8.0)
        h = rng.uniform(2.0, 5.0)
        eye = (rad * np.cos(a), rad * np.sin(a), h)
        views.append(pinhole_hitpoints(eye, (0.0, 0.0, 0.5), side, side))
    return concat_queries(views)


def perturbed_copy(field: Field, seed: int = 1, mean_sigma: float = 0.01,
                   spec_lo: float = 0.8, spec_hi: float = 1.2) -> Field:
    """Target field: means jittered by N(0, mean_sigma), spectra scaled by U[lo, hi]."""
    rng = _rng(seed)
    out = field.copy()
    out.mean = _f32(field.mean + rng.normal(0.0, mean_sigma, field.mean.shape))
    out.spectrum = _f32(field.spectrum * rng.uniform(spec_lo, spec_hi, field.spectrum.shape))
    return out


def subset_field(field: Field, idx: np.ndarray) -> Field:
    return Field(_f32(field.mean[:, idx]), _f32(field.quat[:, idx]),
                 _f32(field.logscale[:, idx]), _f32(field.spectrum[:, idx]))


def subset_queries(q: Queries, idx: np.ndarray) -> Queries:
    return Queries(
        x=_f32(q.x[:, idx]), n=_f32(q.n[:, idx]), wo=_f32(q.wo[:, idx]),
        albedo=None if q.albedo is None else _f32(q.albedo[:, idx]),
        valid=None if q.valid is None else np.ascontiguousarray(q.valid[idx]),
        view_offsets=np.array([0, len(idx)], dtype=np.int64),
    )
