"""One optimisation step of the Gaussian Photon Field over a batch of hit
points, eager or as a captured CUDA graph.

The hit points of any number of views (of any sizes) are one `Queries`
batch, so one index build, one persistent forward and one persistent
backward cover all of them (the loss is the MSE over the batch's valid
points, Sec. 4.3; Adam per Sec. A.2). Every buffer is allocated up front and
the Adam update count lives on the device, so the whole step can be captured
once with `capture()` and replayed: a replay launches the recorded kernels
without any host work.
"""

from __future__ import annotations

from typing import Optional

import torch

from . import api
from .api import (GPF_SUM, PAPER_EPS, PAPER_LR, PAPER_R, AdamState, Field, Index, Queries)


class TrainStep:
    """build index -> radiance forward -> MSE gradient -> radiance backward
    -> Adam, over preallocated buffers.

    field    float32 parameters (updated in place by every step)
    queries  the batch of hit points (all views concatenated)
    target   [C, M] radiance to fit
    index    an Index with capacity for the field and queries (setup_index),
             created for the storage the step reads (see `store`)
    store    None: the pair loops read `field` itself. A GPF_BF16 Field
             (Field.quantized()): the pair loops read this 16-bit copy, the
             gradients (with respect to its decoded values) update the
             float32 master `field`, which is then re-quantised into it.
    """

    def __init__(self, field: Field, queries: Queries, target: torch.Tensor, index: Index,
                 mode: int = GPF_SUM, r_max: float = PAPER_R, eps: float = PAPER_EPS,
                 lr=PAPER_LR, grad_hook=None, store: Optional[Field] = None):
        self.field, self.queries, self.target, self.index = field, queries, target, index
        self.store = store
        self.mode, self.r_max, self.eps, self.lr = mode, r_max, eps, lr
        c, m = field.channels, queries.m
        dev = field.mean.device
        self.state = AdamState.zeros_like(field, device_counter=True)
        self.grads = Field.zeros_like(field)            # float32, like the master
        self.out = torch.empty((c, m), dtype=torch.float32, device=dev)
        self.z = torch.empty((m,), dtype=torch.float32, device=dev)
        self.gout = torch.empty((c, m), dtype=torch.float32, device=dev)
        self.loss = torch.zeros((1,), dtype=torch.float32, device=dev)
        self.mse_ws = api.gpf_mse_workspace(m, dev)
        # device flags of each step's build (GPF_FLAG_*: 0 = usable), copied
        # to pinned host memory at the end of the step, so that a caller can
        # check a replayed step without synchronising the stream
        self.flags = torch.zeros((1,), dtype=torch.int32, device=dev)
        self.flags_host = torch.zeros((1,), dtype=torch.int32).pin_memory()
        self.done = torch.cuda.Event()
        self.grad_hook = grad_hook        # e.g. a data-parallel gradient all-reduce
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    def run_eager(self) -> None:
        """One step, launched now on the current stream."""
        q = self.queries
        f = self.store if self.store is not None else self.field
        self.index.build(f, q)
        self.index.flags_async(self.flags)
        api.gpf_radiance_fwd(self.index, f, q, self.mode, r_max=self.r_max, eps=self.eps,
                             out=self.out, z=self.z)
        api.gpf_mse_loss_grad(self.out, self.target, q.valid, loss=self.loss, grad=self.gout,
                              workspace=self.mse_ws)
        api.gpf_radiance_bwd(self.index, f, q, self.gout, self.out, self.z, self.mode,
                             r_max=self.r_max, eps=self.eps, grads=self.grads)
        if self.grad_hook is not None:
            self.grad_hook(self.grads)
        # an unusable build (a full pair buffer, a sort that gave up, a
        # non-finite parameter) leaves the gradients unwritten: the guard
        # cancels the update on the device
        api.gpf_adam_step(self.field, self.grads, self.state, lr=self.lr, guard=self.index)
        if self.store is not None:
            self.field.quantize_into(self.store)
        self.flags_host.copy_(self.flags, non_blocking=True)

    def capture(self, warmup: int = 1) -> None:
        """Run `warmup` real steps on a side stream (first-use set-up outside
        the capture), then record one step as a CUDA graph without running
        it. Later calls replay the graph."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self.run_eager()
        torch.cuda.current_stream().wait_stream(side)
        self.index.set_timing_events()          # no event records inside the graph
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run_eager()
        self.graph = g

    def __call__(self) -> None:
        if self.graph is not None:
            self.graph.replay()
        else:
            self.run_eager()
        self.done.record()

    def last_flags(self) -> Optional[int]:
        """GPF_FLAG_* bits of the last step's build (0: it was usable and
        the step was applied; else the step left the parameters as they
        were), or None while that step is still running. Never blocks."""
        if not self.done.query():
            return None
        return int(self.flags_host[0])

    def updates(self) -> int:
        """Adam updates applied so far (synchronises)."""
        return self.state.updates()

    def loss_value(self) -> float:
        """The loss of the last step's forward (synchronises)."""
        return float(self.loss.item())


def per_view_step(field: Field, views, targets, indexes, state: AdamState, grads: Field,
                  outs, zs, gouts, mode: int = GPF_SUM, r_max: float = PAPER_R,
                  eps: float = PAPER_EPS, lr=PAPER_LR) -> None:
    """The same step with one launch sequence per view (the baseline the
    batched step is compared with): per view an index build, a forward, its
    MSE gradient and a backward that accumulates into grads; then one Adam
    update. Each view's MSE is normalised by its own valid points."""
    for k, (q, t, idx) in enumerate(zip(views, targets, indexes)):
        idx.build(field, q)
        api.gpf_radiance_fwd(idx, field, q, mode, r_max=r_max, eps=eps, out=outs[k], z=zs[k])
        api.gpf_mse_loss_grad(outs[k], t, q.valid, grad=gouts[k])
        api.gpf_radiance_bwd(idx, field, q, gouts[k], outs[k], zs[k], mode, r_max=r_max, eps=eps,
                             grads=grads, accumulate=k > 0)
    api.gpf_adam_step(field, grads, state, lr=lr)


__all__ = ["TrainStep", "per_view_step"]
