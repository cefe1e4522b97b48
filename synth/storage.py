"""The GPF_BF16 storage form of a field, on the host: an encoder and a
decoder written from the format's definition (16 consecutive Gaussians share
a float32 anchor: the midpoint of their per-axis mean range and of their
log-scale range; the stored values are float32 offsets or values rounded to
the nearest bfloat16, ties to even). Tests use it to give the oracle decoded
parameters that never pass through the CUDA path. No radiance arithmetic."""

from __future__ import annotations

import dataclasses

import numpy as np

from .scenes import Field, _morton_keys

GROUP = 16


def f32_to_bf16(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bits (uint16), round to nearest, ties to even."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = u + 0x7FFF + ((u >> 16) & 1)
    return ((u >> 16) & 0xFFFF).astype(np.uint16)


def bf16_to_f32(h: np.ndarray) -> np.ndarray:
    return (np.asarray(h, dtype=np.uint32) << 16).view(np.float32)


@dataclasses.dataclass
class BF16Field:
    mean: np.ndarray       # uint16 [3,N] offsets from the group origin (float32
                           # means themselves in the float32-mean form)
    quat: np.ndarray       # uint16 [4,N]
    logscale: np.ndarray   # uint16 [3,N] offsets from the group reference
    spectrum: np.ndarray   # uint16 [C,N]
    anchor: np.ndarray     # float32 [ceil(N/16), 4]: origin x, y, z, l_ref


def encode(f: Field, mean32: bool = False) -> BF16Field:
    n = f.mean.shape[1]
    g = (n + GROUP - 1) // GROUP
    pad = g * GROUP - n
    mean = np.pad(f.mean.astype(np.float32), ((0, 0), (0, pad)), constant_values=np.nan)
    lsc = np.pad(f.logscale.astype(np.float32), ((0, 0), (0, pad)), constant_values=np.nan)
    mg = mean.reshape(3, g, GROUP)
    lg = lsc.reshape(3, g, GROUP).transpose(1, 0, 2).reshape(g, 3 * GROUP)
    half = np.float32(0.5)
    origin = ((np.nanmin(mg, axis=2) + np.nanmax(mg, axis=2)) * half).astype(np.float32)   # [3,g]
    lref = ((np.nanmin(lg, axis=1) + np.nanmax(lg, axis=1)) * half).astype(np.float32)     # [g]
    grp = np.arange(n) // GROUP
    anchor = np.stack([origin[0], origin[1], origin[2], lref], axis=1).astype(np.float32)
    mo = (f.mean.astype(np.float32) - origin[:, grp]).astype(np.float32)
    lo = (f.logscale.astype(np.float32) - lref[grp][None, :]).astype(np.float32)
    mean_arr = f.mean.astype(np.float32).copy() if mean32 else f32_to_bf16(mo)
    return BF16Field(mean_arr, f32_to_bf16(f.quat), f32_to_bf16(lo),
                     f32_to_bf16(f.spectrum), anchor)


def decode(b: BF16Field) -> Field:
    n = b.mean.shape[1]
    grp = np.arange(n) // GROUP
    a = b.anchor[grp].T.astype(np.float32)                  # [4,N]
    if b.mean.dtype == np.float32:
        mean = b.mean.copy()
    else:
        mean = (a[:3] + bf16_to_f32(b.mean)).astype(np.float32)
    lsc = (a[3:4] + bf16_to_f32(b.logscale)).astype(np.float32)
    return Field(mean=mean, quat=bf16_to_f32(b.quat).copy(), logscale=lsc,
                 spectrum=bf16_to_f32(b.spectrum).copy())


def morton_order(f: Field) -> np.ndarray:
    """Permutation that sorts the Gaussians by the Morton code of their means
    (stable): consecutive Gaussians, hence anchor groups, are close in space."""
    return np.argsort(_morton_keys(f.mean.T.astype(np.float64)), kind="stable")


def permuted(f: Field, perm: np.ndarray) -> Field:
    return Field(mean=np.ascontiguousarray(f.mean[:, perm]),
                 quat=np.ascontiguousarray(f.quat[:, perm]),
                 logscale=np.ascontiguousarray(f.logscale[:, perm]),
                 spectrum=np.ascontiguousarray(f.spectrum[:, perm]))
