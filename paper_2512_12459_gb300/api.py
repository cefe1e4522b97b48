"""Python binding of libgpf with the same names as the C ABI.

PyTorch supplies device memory and streams; every step of the radiance path
runs in libgpf's CUDA kernels. The functions here only check tensor
properties and marshal pointers."""

from __future__ import annotations

import ctypes
import dataclasses
import math
from typing import Optional, Sequence

import torch

from . import _abi
from ._abi import (GPF_DISK_KDE, GPF_NB_BALL_KNN, GPF_NB_KSIGMA, GPF_NORMALIZED, GPF_SUM,
                   GPFError, check, load)

__all__ = [
    "GPF_SUM", "GPF_NORMALIZED", "GPF_DISK_KDE", "GPFError", "GridConfig", "Field", "Queries", "Index",
    "grid_for_bounds", "gpf_radiance_fwd", "gpf_radiance_bwd", "gpf_mse_loss_grad",
    "gpf_mse_workspace",
    "gpf_adam_step", "AdamState", "PAPER_R", "PAPER_EPS", "PAPER_LR",
]

# Hyper-parameters the paper prints (Sec. A.2 and the query listing of Algorithm S3).
PAPER_R = 0.02
PAPER_EPS = 1e-6
PAPER_LR = 5e-4


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _need(t: torch.Tensor, name: str, rows: int, count: int, dtype=torch.float32):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    want = (rows, count) if rows else (count,)
    if tuple(t.shape) != want:
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {want}")


@dataclasses.dataclass
class Field:
    """N Gaussians as CUDA tensors [rows, N]: mean [3,N], quat [4,N] (w,x,y,z),
    logscale [3,N], spectrum [C,N]. float32 (GPF_F32 storage), or bfloat16
    with `anchor` float32 [ceil(N/16), 4] (GPF_BF16 storage: means and
    log-scales as offsets from each group's anchor; GPF_BF16_MEAN32: the
    same with float32 means; see include/gpf.h)."""

    mean: torch.Tensor
    quat: torch.Tensor
    logscale: torch.Tensor
    spectrum: torch.Tensor
    anchor: Optional[torch.Tensor] = None

    @property
    def n(self) -> int:
        return int(self.mean.shape[1])

    @property
    def channels(self) -> int:
        return int(self.spectrum.shape[0])

    @property
    def storage(self) -> int:
        if self.quat.dtype != torch.bfloat16:
            return _abi.GPF_F32
        return _abi.GPF_BF16 if self.mean.dtype == torch.bfloat16 else _abi.GPF_BF16_MEAN32

    def c_struct(self) -> _abi.gpf_field:
        n, c = self.n, self.channels
        st = self.storage
        dt = torch.float32 if st == _abi.GPF_F32 else torch.bfloat16
        _need(self.mean, "mean", 3, n, torch.bfloat16 if st == _abi.GPF_BF16 else torch.float32)
        _need(self.quat, "quat", 4, n, dt)
        _need(self.logscale, "logscale", 3, n, dt)
        _need(self.spectrum, "spectrum", c, n, dt)
        if st != _abi.GPF_F32 and n > 0:
            _need(self.anchor, "anchor", (n + _abi.GPF_BF16_GROUP - 1) // _abi.GPF_BF16_GROUP, 4)
        return _abi.gpf_field(n, c, self.storage, _ptr(self.mean), _ptr(self.quat),
                              _ptr(self.logscale), _ptr(self.spectrum), _ptr(self.anchor))

    def tensors(self):
        return [self.mean, self.quat, self.logscale, self.spectrum]

    @staticmethod
    def zeros_like(f: "Field") -> "Field":
        return Field(*(torch.zeros_like(t) for t in f.tensors()))

    @staticmethod
    def from_numpy(f, device="cuda") -> "Field":
        return Field(*(torch.as_tensor(a, dtype=torch.float32, device=device).contiguous()
                       for a in (f.mean, f.quat, f.logscale, f.spectrum)))

    @staticmethod
    def empty_bf16(n: int, channels: int, device="cuda", mean32: bool = False) -> "Field":
        """Uninitialised GPF_BF16 (or GPF_BF16_MEAN32) arrays for n Gaussians."""
        g = (n + _abi.GPF_BF16_GROUP - 1) // _abi.GPF_BF16_GROUP
        e = lambda r, dt=torch.bfloat16: torch.empty((r, n), dtype=dt, device=device)  # noqa
        return Field(e(3, torch.float32 if mean32 else torch.bfloat16), e(4), e(3), e(channels),
                     torch.empty((g, 4), dtype=torch.float32, device=device))

    def quantize_into(self, dst: "Field", stream=None) -> "Field":
        """gpf_field_quantize: write the GPF_BF16 form of this float32 field into dst."""
        fs, ds = self.c_struct(), dst.c_struct()
        check(load().gpf_field_quantize(ctypes.byref(fs), ctypes.byref(ds), _stream(stream)),
              "gpf_field_quantize")
        return dst

    def quantized(self, mean32: bool = False, stream=None) -> "Field":
        """A new GPF_BF16 (mean32: GPF_BF16_MEAN32) field holding this float32
        field's quantised form."""
        return self.quantize_into(
            Field.empty_bf16(self.n, self.channels, self.mean.device, mean32), stream)

    def decoded(self) -> "Field":
        """float32 values of a GPF_BF16 field (host-side set-up and checks
        only; the library decodes on the GPU inside gpf_build_index)."""
        if self.storage == _abi.GPF_F32:
            return self
        grp = torch.arange(self.n, device=self.mean.device) // _abi.GPF_BF16_GROUP
        a = self.anchor[grp].T                         # [4, N]
        mean = self.mean if self.storage == _abi.GPF_BF16_MEAN32 else a[:3] + self.mean.float()
        return Field(mean.contiguous(), self.quat.float(),
                     (a[3:4] + self.logscale.float()).contiguous(), self.spectrum.float())


def photon_field(position: torch.Tensor, flux: torch.Tensor, radius: float,
                 cutoff_sigma: float = 3.0) -> Field:
    """Photons as a Field for the GPF_DISK_KDE gather: mean = position [3,N],
    spectrum = flux [C,N], identity rotations and isotropic log-scales
    log(radius / cutoff_sigma), so that each photon's k-sigma box is the box
    of its gather disk."""
    n = int(position.shape[1])
    quat = torch.zeros((4, n), dtype=torch.float32, device=position.device)
    quat[0] = 1.0
    lsc = torch.full((3, n), math.log(radius / cutoff_sigma), dtype=torch.float32,
                     device=position.device)
    return Field(position.float().contiguous(), quat, lsc, flux.float().contiguous())


@dataclasses.dataclass
class Queries:
    """M hit points as CUDA tensors: x, normal, wo [3,M] float32; albedo [C,M]
    float32 or None; valid [M] uint8 or None."""

    x: torch.Tensor
    normal: torch.Tensor
    wo: torch.Tensor
    albedo: Optional[torch.Tensor] = None
    valid: Optional[torch.Tensor] = None

    @property
    def m(self) -> int:
        return int(self.x.shape[1])

    def c_struct(self, channels: Optional[int] = None) -> _abi.gpf_queries:
        m = self.m
        _need(self.x, "x", 3, m)
        _need(self.normal, "normal", 3, m)
        _need(self.wo, "wo", 3, m)
        if self.albedo is not None:
            _need(self.albedo, "albedo", channels or int(self.albedo.shape[0]), m)
        if self.valid is not None:
            _need(self.valid, "valid", 0, m, torch.uint8)
        return _abi.gpf_queries(m, _ptr(self.x), _ptr(self.normal), _ptr(self.wo),
                                _ptr(self.albedo), _ptr(self.valid))

    @staticmethod
    def from_numpy(q, device="cuda") -> "Queries":
        t = lambda a, dt=torch.float32: None if a is None else torch.as_tensor(  # noqa: E731
            a, dtype=dt, device=device).contiguous()
        return Queries(t(q.x), t(q.n), t(q.wo), t(q.albedo), t(q.valid, torch.uint8))


@dataclasses.dataclass
class GridConfig:
    """Multi-level grid and capacities of an index (gpf_grid_config): level L
    has cells of edge cell_size * 2^L; hit points are sorted on query_level,
    a dims grid; Gaussian lists live in 2^hash_bits buckets."""

    origin: Sequence[float]
    cell_size: float
    levels: int
    max_span: int
    query_level: int
    dims: Sequence[int]
    hash_bits: int
    channels: int
    cutoff_sigma: float = 3.0
    max_gaussians: int = 0
    max_queries: int = 0
    max_pairs: int = 0
    brute_force: bool = False
    coop_cells: int = 0        # forward tile shape (0 = library default, 4)
    field_storage: int = 0     # GPF_F32 or GPF_BF16 fields
    ball_radius: float = 0.0   # > 0: centre entries for GPF_NB_BALL_KNN queries
    max_nb_pairs: int = 0      # capacity of the GPF_NB_BALL_KNN backward's pairs
    split_items: int = 0       # > 0: split forward tiles of more estimated work
    tile_order: int = 0        # hit points inside a query cell by 2^b sub-cells (b = 0..2)

    def c_struct(self) -> _abi.gpf_grid_config:
        return _abi.gpf_grid_config((ctypes.c_float * 3)(*self.origin), float(self.cell_size),
                                    int(self.levels), int(self.max_span), int(self.query_level),
                                    (ctypes.c_int32 * 3)(*[int(d) for d in self.dims]),
                                    int(self.hash_bits), int(self.channels),
                                    float(self.cutoff_sigma), 1 if self.brute_force else 0,
                                    int(self.coop_cells), int(self.field_storage),
                                    float(self.ball_radius), int(self.max_gaussians),
                                    int(self.max_queries),
                                    int(self.max_pairs), int(self.max_nb_pairs),
                                    int(self.split_items), int(self.tile_order))


def grid_for_bounds(lo: Sequence[float], hi: Sequence[float], cell_size: float, channels: int,
                    max_gaussians: int, max_queries: int, max_pairs: int,
                    cutoff_sigma: float = 3.0, levels: int = 1, max_span: int = 4,
                    query_level: int = 0, hash_bits: int = 20) -> GridConfig:
    """A grid whose query level covers [lo, hi] with cells of cell_size *
    2^query_level (points outside are clamped into the border cells, which
    stays exact)."""
    cq = cell_size * (1 << query_level)
    dims = [max(1, min(_abi.GPF_MAX_DIM, int(math.ceil((float(h) - float(l)) / cq))))
            for l, h in zip(lo, hi)]
    return GridConfig([float(v) for v in lo], cell_size, levels, max_span, query_level, dims,
                      hash_bits, channels, cutoff_sigma, max_gaussians, max_queries, max_pairs)


class Index:
    """gpf_index handle plus the device workspace it lives in (a uint8 CUDA
    tensor owned by this object)."""

    def __init__(self, grid: GridConfig, device="cuda"):
        lib = load()
        self._lib = lib
        self.grid = grid
        self._cfg = grid.c_struct()
        h = ctypes.c_void_p()
        check(lib.gpf_index_create(ctypes.byref(self._cfg), ctypes.byref(h)), "gpf_index_create")
        self._h = h
        sz = ctypes.c_size_t()
        check(lib.gpf_index_workspace_size(h, ctypes.byref(sz)), "gpf_index_workspace_size")
        self.workspace_bytes = int(sz.value)
        self.workspace = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8,
                                     device=device)
        self._field = None
        self._queries = None

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.gpf_index_destroy(h)
            self._h = None

    def build(self, field: Field, queries: Queries, stream=None) -> None:
        """gpf_build_index for (field, queries)."""
        fs = field.c_struct()
        qs = queries.c_struct(field.channels)
        check(self._lib.gpf_build_index(self._h, ctypes.byref(fs), ctypes.byref(qs),
                                        self.workspace.data_ptr(), self.workspace_bytes,
                                        _stream(stream)), "gpf_build_index")
        self._field, self._queries = field, queries

    def set_timing_events(self, fwd=None, bwd=None) -> None:
        """gpf_index_set_timing_events: `fwd` and `bwd` are (start, stop)
        pairs of torch.cuda.Event (enable_timing=True) or None; later
        gpf_radiance_fwd / gpf_radiance_bwd calls record them around their
        pair-loop kernels."""
        hs = []
        for pair in (fwd, bwd):
            for ev in (pair if pair is not None else (None, None)):
                hs.append(_event_handle(ev))
        self._timing = (fwd, bwd)   # keep the events alive while they are set
        check(self._lib.gpf_index_set_timing_events(self._h, *hs), "gpf_index_set_timing_events")

    def stats(self, stream=None, raise_on_flags: bool = False) -> dict:
        """gpf_index_stats (synchronises the stream): the counters of the last
        build and its device flags (GPF_FLAG_* bits in "flags"; "overflow"
        is the capacity bit). A set flag raises GPFError only with
        raise_on_flags; other failures always raise."""
        st = _abi.gpf_index_stats_t()
        status = self._lib.gpf_index_stats(self._h, ctypes.byref(st), _stream(stream))
        out = {"n_pairs": st.n_pairs, "n_active": st.n_active, "n_live": st.n_live,
               "n_small": st.n_small, "n_huge": st.n_huge, "n_split": st.n_split,
               "level_mask": st.level_mask, "flags": st.flags, "overflow": bool(st.overflow),
               "n_hybrid_units": st.n_hybrid_units, "n_nb_pairs": st.n_nb_pairs}
        flag_status = (_abi.GPF_ERR_CAPACITY, _abi.GPF_ERR_TIMEOUT, _abi.GPF_ERR_NONFINITE)
        if status != _abi.GPF_OK and (raise_on_flags or status not in flag_status):
            check(status, "gpf_index_stats")
        return out

    def flags_async(self, flags: torch.Tensor, stream=None) -> None:
        """gpf_index_flags_async: enqueue a write of the last build's device
        flags (GPF_FLAG_* bits, 0 = usable) into `flags`, a 1-element int32
        CUDA tensor, without synchronising."""
        if flags.dtype != torch.int32 or not flags.is_cuda or flags.numel() < 1:
            raise ValueError("flags must be an int32 CUDA tensor with at least one element")
        check(self._lib.gpf_index_flags_async(self._h, flags.data_ptr(), _stream(stream)),
              "gpf_index_flags_async")


def _event_handle(ev):
    """The cudaEvent_t of a torch.cuda.Event (created on first use), or None."""
    if ev is None:
        return None
    h = int(ev.cuda_event or 0)
    if h == 0:
        ev.record()          # torch creates the CUDA event lazily
        h = int(ev.cuda_event)
    return h


def _params(mode, r_max, eps, neighbourhood=0, ball_r=0.0, k_min=0,
            f64_sums=False) -> _abi.gpf_query_params:
    return _abi.gpf_query_params(int(mode), float(r_max), float(eps), int(neighbourhood),
                                 float(ball_r), int(k_min), 1 if f64_sums else 0)


def gpf_radiance_fwd(index: Index, field: Field, queries: Queries, mode: int = GPF_SUM,
                     r_max: float = math.inf, eps: float = PAPER_EPS,
                     out: Optional[torch.Tensor] = None, z: Optional[torch.Tensor] = None,
                     want_z: bool = True, stream=None, neighbourhood: int = 0,
                     ball_r: float = PAPER_R, k_min: int = 3):
    """Radiance O [C,M] (and Z [M]) at the hit points the index was built for.
    neighbourhood GPF_NB_KSIGMA (default): the index's k-sigma ellipsoids;
    GPF_NB_BALL_KNN: the paper's ball(ball_r) or k_min nearest means (the
    index needs ball_radius >= ball_r)."""
    m, c = queries.m, field.channels
    dev = queries.x.device
    if out is None:
        out = torch.empty((c, m), dtype=torch.float32, device=dev)
    if z is None and want_z:
        z = torch.empty((m,), dtype=torch.float32, device=dev)
    _need(out, "out", c, m)
    if z is not None:
        _need(z, "z", 0, m)
    fs, qs = field.c_struct(), queries.c_struct(c)
    ps = _params(mode, r_max, eps, neighbourhood, ball_r, k_min)
    check(index._lib.gpf_radiance_fwd(index.handle, ctypes.byref(fs), ctypes.byref(qs),
                                      ctypes.byref(ps), out.data_ptr(), _ptr(z),
                                      _stream(stream)), "gpf_radiance_fwd")
    return out, z


def gpf_count_pairs(index: Index, field: Field, queries: Queries, stream=None) -> dict:
    """Pairs the forward evaluates after culling ("candidates") and pairs with
    Q <= k^2 ("included"); synchronises the stream to read them."""
    counts = torch.zeros(2, dtype=torch.int64, device=queries.x.device)
    fs, qs = field.c_struct(), queries.c_struct(field.channels)
    check(index._lib.gpf_count_pairs(index.handle, ctypes.byref(fs), ctypes.byref(qs),
                                     counts.data_ptr(), _stream(stream)), "gpf_count_pairs")
    c = counts.cpu().tolist()
    return {"candidates": int(c[0]), "included": int(c[1])}


def gpf_measure_alu_peak(which: int = _abi.GPF_PEAK_FP32_FMA, iters: int = 4096) -> dict:
    """gpf_measure_alu_peak: measured FP32 FMA flop/s (which=GPF_PEAK_FP32_FMA)
    or ex2 results/s (GPF_PEAK_EX2) of the current device (synchronous)."""
    rate, sec = ctypes.c_double(), ctypes.c_double()
    check(load().gpf_measure_alu_peak(int(which), int(iters), ctypes.byref(rate),
                                      ctypes.byref(sec)), "gpf_measure_alu_peak")
    return {"per_second": float(rate.value), "seconds": float(sec.value)}


def gpf_launch_count() -> int:
    """Kernels libgpf has launched in this process."""
    return int(load().gpf_launch_count())


def gpf_radiance_bwd(index: Index, field: Field, queries: Queries, grad_out: torch.Tensor,
                     out: Optional[torch.Tensor] = None, z: Optional[torch.Tensor] = None,
                     mode: int = GPF_SUM, r_max: float = math.inf, eps: float = PAPER_EPS,
                     grads: Optional[Field] = None, accumulate: bool = False,
                     stream=None, neighbourhood: int = 0, f64_sums: bool = False,
                     ball_r: float = PAPER_R, k_min: int = 3) -> Field:
    """Gradients (a Field of tensors) of sum(grad_out * O) w.r.t. mean, quat,
    logscale and spectrum, for the neighbourhood of the forward
    (GPF_NB_KSIGMA, or GPF_NB_BALL_KNN with ball_r and k_min on an index with
    max_nb_pairs > 0). f64_sums=True runs the float64 gradient-check build of
    the per-Gaussian sums (gpf_query_params.f64_sums)."""
    m, c = queries.m, field.channels
    _need(grad_out, "grad_out", c, m)
    if grads is None:       # float32 gradients for either storage
        mk = torch.zeros if accumulate else torch.empty
        grads = Field(*(mk(tuple(t.shape), dtype=torch.float32, device=t.device)
                        for t in field.tensors()))
    for name, g, t in zip(("grad_mean", "grad_quat", "grad_logscale", "grad_spectrum"),
                          grads.tensors(), field.tensors()):
        _need(g, name, t.shape[0], t.shape[1])
    if mode == GPF_NORMALIZED:
        if out is None or z is None:
            raise ValueError("GPF_NORMALIZED backward needs the forward's out and z")
        _need(out, "out", c, m)
        _need(z, "z", 0, m)
    fs, qs = field.c_struct(), queries.c_struct(c)
    ps = _params(mode, r_max, eps, neighbourhood, ball_r, k_min, f64_sums=f64_sums)
    gs = _abi.gpf_field_grad(_ptr(grads.mean), _ptr(grads.quat), _ptr(grads.logscale),
                             _ptr(grads.spectrum), 1 if accumulate else 0, 0)
    check(index._lib.gpf_radiance_bwd(index.handle, ctypes.byref(fs), ctypes.byref(qs),
                                      ctypes.byref(ps), grad_out.data_ptr(), _ptr(out), _ptr(z),
                                      ctypes.byref(gs), _stream(stream)), "gpf_radiance_bwd")
    return grads


def gpf_sort_pairs(keys: torch.Tensor, vals: torch.Tensor, bits: int = 32, check_wait: bool = True,
                   stream=None):
    """The index build's stable radix sort of uint32 (key, value) pairs by key
    bits [0, bits), as int32 CUDA tensors of one length (bit patterns of
    uint32). Returns new (keys, vals) tensors in key order, equal keys in
    input order. check_wait=True synchronises and raises GPFError
    (GPF_ERR_TIMEOUT) if a bounded wait of the sort gave up."""
    n = int(keys.numel())
    for t, name in ((keys, "keys"), (vals, "vals")):
        if t.dtype != torch.int32 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name}: contiguous int32 CUDA tensor of {n} elements expected")
    lib = load()
    sz = ctypes.c_size_t()
    check(lib.gpf_sort_pairs_workspace_size(n, ctypes.byref(sz)), "gpf_sort_pairs_workspace_size")
    ws = torch.empty(int(sz.value), dtype=torch.uint8, device=keys.device)
    k0, v0 = keys.clone(), vals.clone()
    k1, v1 = torch.empty_like(k0), torch.empty_like(v0)
    alt = ctypes.c_int32()
    check(lib.gpf_sort_pairs(k0.data_ptr(), v0.data_ptr(), k1.data_ptr(), v1.data_ptr(), n, bits,
                             ws.data_ptr(), ws.numel(), ctypes.byref(alt), _stream(stream)),
          "gpf_sort_pairs")
    if check_wait:
        check(lib.gpf_sort_pairs_check(ws.data_ptr(), _stream(stream)), "gpf_sort_pairs_check")
    return (k1, v1) if alt.value else (k0, v0)


class _MseWorkspace:
    """Scratch of gpf_mse_loss_grad, one buffer per (size, device, stream).
    Each buffer is allocated while its stream is current, so PyTorch's caching
    allocator hands its memory to another tensor only after the work queued
    on that stream has used it; calls on different streams never share one."""
    cache = {}
    max_entries = 16

    @classmethod
    def get(cls, m: int, device, stream) -> torch.Tensor:
        key = (m, str(device), stream.cuda_stream)
        ws = cls.cache.get(key)
        if ws is None:
            sz = ctypes.c_size_t()
            check(load().gpf_mse_workspace_size(m, ctypes.byref(sz)), "gpf_mse_workspace_size")
            with torch.cuda.stream(stream):
                ws = torch.empty(max(int(sz.value), 256), dtype=torch.uint8, device=device)
            if len(cls.cache) >= cls.max_entries:
                cls.cache.pop(next(iter(cls.cache)))
            cls.cache[key] = ws
        return ws


def gpf_mse_workspace(m: int, device="cuda") -> torch.Tensor:
    """A device scratch buffer for gpf_mse_loss_grad over m hit points (for
    callers that keep their own, e.g. a step captured as a CUDA graph)."""
    sz = ctypes.c_size_t()
    check(load().gpf_mse_workspace_size(m, ctypes.byref(sz)), "gpf_mse_workspace_size")
    return torch.empty(max(int(sz.value), 256), dtype=torch.uint8, device=device)


def gpf_mse_loss_grad(out: torch.Tensor, target: torch.Tensor,
                      valid: Optional[torch.Tensor] = None, loss: Optional[torch.Tensor] = None,
                      grad: Optional[torch.Tensor] = None, stream=None,
                      workspace: Optional[torch.Tensor] = None):
    """MSE loss (a 1-element CUDA tensor) and its gradient with respect to out.
    workspace: a buffer from gpf_mse_workspace(m), or None for one cached per
    (size, device, stream)."""
    c, m = int(out.shape[0]), int(out.shape[1])
    _need(out, "out", c, m)
    _need(target, "target", c, m)
    if valid is not None:
        _need(valid, "valid", 0, m, torch.uint8)
    if loss is None:
        loss = torch.empty((1,), dtype=torch.float32, device=out.device)
    if grad is None:
        grad = torch.empty_like(out)
    st = stream if stream is not None else torch.cuda.current_stream(out.device)
    ws = workspace if workspace is not None else _MseWorkspace.get(m, out.device, st)
    check(load().gpf_mse_loss_grad(m, c, out.data_ptr(), target.data_ptr(), _ptr(valid),
                                   loss.data_ptr(), grad.data_ptr(), ws.data_ptr(), ws.numel(),
                                   st.cuda_stream), "gpf_mse_loss_grad")
    return loss, grad


@dataclasses.dataclass
class AdamState:
    """First and second moments and the update count. With `step_counter`
    (a device int64 tensor, see `with_device_counter`) the count lives on the
    device: each update reads and increments it, which is what a captured
    CUDA graph of the training step needs; `step` is then not advanced."""
    m: Field
    v: Field
    step: int = 0
    step_counter: Optional[torch.Tensor] = None

    @staticmethod
    def zeros_like(f: Field, device_counter: bool = False) -> "AdamState":
        ctr = torch.zeros(1, dtype=torch.int64, device=f.mean.device) if device_counter else None
        return AdamState(Field.zeros_like(f), Field.zeros_like(f), 0, ctr)

    def updates(self) -> int:
        """Updates applied so far (reads the device counter when there is one)."""
        return int(self.step_counter.item()) if self.step_counter is not None else self.step


def _grad_struct(f: Field) -> _abi.gpf_field_grad:
    return _abi.gpf_field_grad(_ptr(f.mean), _ptr(f.quat), _ptr(f.logscale), _ptr(f.spectrum), 0, 0)


def gpf_adam_step(params: Field, grads: Field, state: AdamState, lr=PAPER_LR, beta1: float = 0.9,
                  beta2: float = 0.999, eps: float = 1e-8, stream=None,
                  guard: Optional[Index] = None) -> None:
    """One Adam update of params in place; state.step is incremented first
    (host count). guard: an Index whose last build, if it set a device flag,
    cancels the update on the device (parameters, moments and the device
    step counter stay as they were)."""
    lrs = list(lr) if isinstance(lr, (list, tuple)) else [float(lr)] * 4
    for g, p in zip(grads.tensors() + state.m.tensors() + state.v.tensors(), params.tensors() * 3):
        _need(g, "adam tensor", p.shape[0], p.shape[1])
    fs = params.c_struct()
    if state.step_counter is not None:
        hp = _abi.gpf_adam_hparams((ctypes.c_float * 4)(*lrs), beta1, beta2, eps, 0,
                                   state.step_counter.data_ptr(),
                                   guard.handle if guard is not None else None)
    else:
        state.step += 1
        hp = _abi.gpf_adam_hparams((ctypes.c_float * 4)(*lrs), beta1, beta2, eps, state.step,
                                   None, guard.handle if guard is not None else None)
    g, m, v = _grad_struct(grads), _grad_struct(state.m), _grad_struct(state.v)
    check(load().gpf_adam_step(ctypes.byref(fs), ctypes.byref(g), ctypes.byref(m),
                               ctypes.byref(v), ctypes.byref(hp), _stream(stream)),
          "gpf_adam_step")
