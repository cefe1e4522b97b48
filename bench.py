"""Benchmark of the Gaussian Photon Field hit-point radiance path on GB300.

One step = the whole hot path over one batch of hit points:
    gpf_build_index -> gpf_radiance_fwd -> gpf_mse_loss_grad
    -> gpf_radiance_bwd -> gpf_adam_step
on the paper-scale synthetic workload: 1,000,000 Gaussians from a caustic-like
photon map on an analytic floor + sphere scene, one 1024 x 1024 pinhole view
(hit points by analytic ray intersection), 3-sigma truncation, falloff radius
r = 0.02, MSE against a target rendered from a perturbed copy of the field,
Adam with lr 5e-4.

Prints one JSON line. --impl reference times the FP64 CPU oracle instead.
Multi-GPU (torchrun): every rank renders its own view of the same field and
the gradients are summed over ranks before the Adam step.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_PHOTONS = 1_000_000
VIEW = 1024
R_MAX = 0.02
CUTOFF = 3.0
CELL = 0.02          # edge of the hit-point grid cells the planner aims for
LR = 5e-4
EYE0 = (0.0, -6.0, 4.0)
LOOK_AT = (0.0, 0.0, 0.5)
L2_BYTES = 129 * 1024 * 1024
METRIC = "hit-point radiance queries/sec (fwd, fwd+bwd) at 1M Gaussians; % of HBM/SFU roofline"
WORKLOAD = "caustic floor+sphere scene, 1,000,000 Gaussians, 1024x1024 view, 3-sigma grid, r=0.02"


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def view_eye(rank: int):
    """Rank 0 uses the reference camera; other ranks orbit it in azimuth."""
    if rank == 0:
        return EYE0
    a = -math.pi / 2 + rank * (2 * math.pi / 8)
    return (6.0 * math.cos(a), 6.0 * math.sin(a), 4.0)


def make_inputs(rank: int):
    import synth
    pos, flux = synth.caustic_photons(N_PHOTONS, seed=0)
    fnp = synth.field_from_photons(pos, flux, seed=0)
    tgt = synth.perturbed_copy(fnp, seed=1)
    qnp = synth.pinhole_hitpoints(view_eye(rank), LOOK_AT, VIEW, VIEW)
    return fnp, tgt, qnp


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# DRAM bytes (read + write) per launch of the pair-loop kernels on this
# workload, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum,
# third warm-up step of `python bench.py --steps 3 --warmup 3
# --no-cpu-baseline --grid 0.0307543,3,8,4096`, the grid the autotuner chooses
# for this scene), with the SHA-256 of the sources the kernel was built from;
# reported only while those sources are unchanged.
PROFILED_TRAFFIC = {
    "fwd_kernel": {"bytes": 418877696 + 18759680, "sources": {
        "paper_2512_12459_gb300/csrc/gpf_fwd.cu":
            "5e45c374e582e292bf8246d6b9f27b44299f26c93642e36598cc9f374ff4afbf",
        "paper_2512_12459_gb300/csrc/gpf_common.cuh":
            "06d7c449435ef4ee171339a3ee1cd6637db6f450d660a45c626362deb382a027"}},
    "bwd_grid_kernel": {"bytes": 150179840 + 50914048, "sources": {
        "paper_2512_12459_gb300/csrc/gpf_bwd.cu":
            "8be4d53dbfcaa580cbb42cd7633aa4bf6d73ca2a2583310392b4b649623d85f3",
        "paper_2512_12459_gb300/csrc/gpf_common.cuh":
            "06d7c449435ef4ee171339a3ee1cd6637db6f450d660a45c626362deb382a027"}},
}


def _sha256(path: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, path), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()


def profiled_traffic(kernel: str):
    rec = PROFILED_TRAFFIC.get(kernel)
    if rec is None:
        return None
    if any(_sha256(p) != h for p, h in rec["sources"].items()):
        return None
    return rec["bytes"]


def fp32_peak_tflops(sm_mhz_max: float, sms: int = 152) -> float:
    """FP32 lane peak: SMs x 128 FP32 lanes x 2 flops (FMA) x max SM clock."""
    return sms * 128 * 2 * sm_mhz_max * 1e6 / 1e12


# ---- the FP64 oracle on all host cores (the CPU baseline and --impl reference)
_W = {}


def _oracle_worker_init(mean, quat, logscale, spectrum):
    _W["f"] = (mean, quat, logscale, spectrum)


def _oracle_task(x, n, wo, valid, target):
    """Forward + backward of a few hit points over every Gaussian (the oracle
    as it stands), in a worker process; returns the forward's per-point
    results for the error check."""
    import oracle
    mean, quat, logscale, spectrum = _W["f"]
    fo = oracle.radiance_fwd(mean, quat, logscale, spectrum, x, n, wo, None, valid,
                             r_max=R_MAX, cutoff_sigma=CUTOFF)
    g = oracle.mse_loss_grad(fo["out"], target, valid)
    oracle.radiance_bwd(mean, quat, logscale, spectrum, x, n, wo, g, None, valid,
                        r_max=R_MAX, cutoff_sigma=CUTOFF)
    return {k: fo[k] for k in ("out", "denom", "logw_max", "near_cutoff")}


class OraclePool:
    """A spawn-started pool of one process per host core (os.sched_getaffinity),
    each with one BLAS/OpenMP thread, holding the field. Spawned workers share
    no CUDA state with this process."""

    def __init__(self, fnp):
        import concurrent.futures
        import multiprocessing as mp
        self.cores = len(os.sched_getaffinity(0))
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                 "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"        # inherited by the spawned workers only
        try:
            self.ex = concurrent.futures.ProcessPoolExecutor(
                max_workers=self.cores, mp_context=mp.get_context("spawn"),
                initializer=_oracle_worker_init,
                initargs=(fnp.mean, fnp.quat, fnp.logscale, fnp.spectrum))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self, qnp, tgt_out_fn, budget_s: float, chunk: int = 4, seed: int = 123):
        """Keeps every core busy with `chunk`-point tasks until budget_s has
        passed, then waits for the tasks in flight. Returns (queries/s, points,
        seconds, {point index: forward result})."""
        import concurrent.futures
        rng = np.random.default_rng(seed)
        act = np.flatnonzero(qnp.valid.astype(bool))
        t0 = time.perf_counter()
        pending, results = {}, {}

        def submit():
            sel = rng.choice(act, size=chunk, replace=False)
            fut = self.ex.submit(_oracle_task, qnp.x[:, sel], qnp.n[:, sel], qnp.wo[:, sel],
                                 qnp.valid[sel], tgt_out_fn(sel))
            pending[fut] = sel

        for _ in range(self.cores):
            submit()
        done = 0
        while pending:
            fin, _ = concurrent.futures.wait(list(pending),
                                             return_when=concurrent.futures.FIRST_COMPLETED)
            for fut in fin:
                sel = pending.pop(fut)
                res = fut.result()
                done += len(sel)
                for j, i in enumerate(sel):
                    results[int(i)] = {k: (v[..., j] if np.ndim(v) > 1 else v[j])
                                       for k, v in res.items()}
                if time.perf_counter() - t0 < budget_s:
                    submit()
        dt = time.perf_counter() - t0
        return done / dt, done, dt, results

    def close(self):
        self.ex.shutdown(wait=True)


def error_vs_oracle(out_gpu, results):
    """Relative error |O_gpu - O_ref| / (rho sum w |Phi|) at the oracle's sample
    points (hit points with a pair within 1e-4 of the cutoff excluded, as in
    the parity tests): max, 99th percentile and median over points."""
    errs = []
    for i, r in results.items():
        if r["near_cutoff"]:
            continue
        den = np.maximum(r["denom"], 1e-20)
        errs.append(float(np.max(np.abs(out_gpu[:, i] - r["out"]) / den)))
    if not errs:
        return None
    e = np.asarray(errs)
    return {"max": float(e.max()), "p99": float(np.quantile(e, 0.99)),
            "median": float(np.median(e)), "points": int(e.size),
            "excluded_near_cutoff": int(len(results) - e.size),
            "metric": "per hit point max over channels of |O_gpu - O_oracle| / (rho sum_i w_i "
                      "|Phi_i|), oracle in float64 over all Gaussians"}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle timed on all host cores, each step a
    bounded random sample of the workload's hit points (fwd + bwd of each over
    all Gaussians), sized so that the whole run ends within a few minutes."""
    if rank != 0:
        return
    fnp, tgt, qnp = make_inputs(0)
    tgt_fn = lambda sel: np.zeros((3, len(sel)))  # noqa: E731  (target values do not change the work)
    per_step = min(args.ref_budget, 150.0 / max(1, args.steps + args.warmup))
    pool = OraclePool(fnp)
    steps = []
    for _ in range(args.warmup):
        pool.run(qnp, tgt_fn, budget_s=per_step / 2)
    for k in range(args.steps):
        rate, done, dt, _ = pool.run(qnp, tgt_fn, budget_s=per_step, seed=1000 + k)
        steps.append((rate, done, dt))
    pool.close()
    rate = sum(s[1] for s in steps) / sum(s[2] for s in steps)
    n_active = int(qnp.valid.sum())
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "queries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * n_active / rate, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": n_active, "seq_len": None,
                   "parallelism": "cpu", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": rate, "unit": "queries/s", "cores": pool.cores,
                         "kind": "oracle",
                         "sample": f"{sum(s[1] for s in steps)} random valid hit points in "
                                   f"{args.steps} steps of about {per_step:.1f} s, fwd+bwd each "
                                   "over all 1,000,000 Gaussians (numpy float64, one process "
                                   "per core); ms_per_step extrapolates to the full view"},
        "e2e": {"value": rate, "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Many views of uneven resolution in one batch: the autotuned index, the
    whole step (build, forward, MSE, backward, Adam) captured once as a CUDA
    graph and replayed, against the same step as one launch sequence per view.
    One GPU; inputs (several GB) are larger than L2."""
    import torch
    import synth
    import paper_2512_12459_gb300 as gpf
    from paper_2512_12459_gb300.setup_index import autotune, make_index
    from paper_2512_12459_gb300.train import TrainStep, per_view_step

    torch.cuda.set_device(0)
    t0 = time.time()
    pos, flux = synth.caustic_photons(args.batched_photons, seed=0)
    fnp = synth.field_from_photons(pos, flux, seed=0)
    tgt_np = synth.perturbed_copy(fnp, seed=1)
    qnp = synth.uneven_views(args.batched_views, seed=0)
    gen_s = time.time() - t0
    field = gpf.Field.from_numpy(fnp)
    queries = gpf.Queries.from_numpy(qnp)
    offs = qnp.view_offsets
    n_active = int(qnp.valid.sum())

    tf = gpf.Field.from_numpy(tgt_np)
    tidx = make_index(tf, queries, query_cell=CELL)
    tidx.build(tf, queries)
    target, _ = gpf.gpf_radiance_fwd(tidx, tf, queries, gpf.GPF_SUM, r_max=R_MAX)
    target = target.clone()
    del tidx, tf
    torch.cuda.empty_cache()

    t0 = time.time()
    grid, report = autotune(field, queries, r_max=R_MAX, repeats=4)
    tune_s = time.time() - t0
    idx = make_index(field, queries, grid=grid, headroom=1.25)
    step = TrainStep(field, queries, target, idx, r_max=R_MAX, lr=LR)
    step.capture(warmup=args.warmup)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    launches0 = gpf.gpf_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    e1.synchronize()
    graph_ms = e0.elapsed_time(e1) / args.steps
    graph_launches = gpf.gpf_launch_count() - launches0   # replays launch nothing from the host
    st = idx.stats()
    if st["overflow"]:
        raise RuntimeError(f"pair buffer overflow: {st}")

    # the per-view baseline: one index (capacity of the largest view), one
    # launch sequence per view, the same field and Adam
    views = [gpf.Queries.from_numpy(synth.subset_queries(qnp, np.arange(offs[v], offs[v + 1])))
             for v in range(len(offs) - 1)]
    vt = [target[:, offs[v]:offs[v + 1]].contiguous() for v in range(len(offs) - 1)]
    big = int(np.argmax(np.diff(offs)))
    # a view occupies a subset of the batch's cells: its entries fit the batch's count
    pidx = make_index(field, views[big], grid=grid, max_queries=int(np.diff(offs).max()),
                      max_pairs=int(st["n_pairs"] * 1.25) + 1024)
    pf = gpf.Field(*(t.clone() for t in field.tensors()))
    pstate = gpf.AdamState.zeros_like(pf, device_counter=True)
    pgrads = gpf.Field.zeros_like(pf)
    outs = [torch.empty_like(t) for t in vt]
    zs = [torch.empty((v.m,), device="cuda") for v in views]
    gouts = [torch.empty_like(t) for t in vt]
    pidxs = [pidx] * len(views)
    for _ in range(args.warmup):
        per_view_step(pf, views, vt, pidxs, pstate, pgrads, outs, zs, gouts, r_max=R_MAX, lr=LR)
    torch.cuda.synchronize()
    launches0 = gpf.gpf_launch_count()
    e0.record()
    for _ in range(args.steps):
        per_view_step(pf, views, vt, pidxs, pstate, pgrads, outs, zs, gouts, r_max=R_MAX, lr=LR)
    e1.record()
    e1.synchronize()
    view_ms = e0.elapsed_time(e1) / args.steps
    view_launches = (gpf.gpf_launch_count() - launches0) / args.steps
    if pidx.stats()["overflow"]:
        raise RuntimeError("per-view pair buffer overflow")

    line = {
        "metric": METRIC, "value": n_active / (graph_ms / 1e3), "unit": "queries/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": graph_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{len(offs) - 1} uneven views (sides 256..1024), "
                               f"{fnp.n:,} Gaussians, one batch, CUDA graph",
                   "hit_points": int(qnp.m), "active_hit_points": n_active,
                   "gaussians": fnp.n, "l2": "inputs larger than L2"},
        "per_view": {"value": n_active / (view_ms / 1e3), "ms_per_step": view_ms,
                     "launches_per_step": view_launches},
        "graph_vs_per_view": view_ms / graph_ms,
        "graph_host_launches_per_step": graph_launches / args.steps,
        "autotuned": {"query_cell": grid.cell_size * (1 << grid.query_level),
                      "query_level": grid.query_level, "max_span": grid.max_span,
                      "coop_cells": grid.coop_cells, "split_items": grid.split_items,
                      "levels": grid.levels,
                      "hash_bits": grid.hash_bits},
        "autotune_trials": [[k, round(ms, 3)] for k, ms in report],
        "setup_s": {"generate": round(gen_s, 1), "autotune": round(tune_s, 1)},
        "index": {"n_pairs": st["n_pairs"]},
    }
    print(json.dumps(line), flush=True)


def run_train(args):
    """The training run of the measurement plan's third configuration: the
    1,000,000-Gaussian caustic field fitted, over 8 orbit views of 800 x 800
    (radius 6, height 3, aimed at (0, 0, 1)), to targets rendered from a
    perturbed copy (means + N(0, 0.01), spectra x U[0.8, 1.2]); Adam at lr
    5e-4 for --train-steps steps, each a replay of one captured CUDA graph
    (build, forward, MSE, backward, Adam). Reports time per step and the loss
    curve (the loss of every step copied on the device, read once at the end)."""
    import torch
    import synth
    import paper_2512_12459_gb300 as gpf
    from paper_2512_12459_gb300.setup_index import autotune, make_index
    from paper_2512_12459_gb300.train import TrainStep

    torch.cuda.set_device(0)
    t0 = time.time()
    pos, flux = synth.caustic_photons(N_PHOTONS, seed=0)
    fnp = synth.field_from_photons(pos, flux, seed=0)
    tgt_np = synth.perturbed_copy(fnp, seed=1)
    qnp = synth.orbit_views(8, 800, 800)
    gen_s = time.time() - t0
    field = gpf.Field.from_numpy(fnp)
    queries = gpf.Queries.from_numpy(qnp)
    n_active = int(qnp.valid.sum())
    tf = gpf.Field.from_numpy(tgt_np)
    tidx = make_index(tf, queries, query_cell=CELL)
    tidx.build(tf, queries)
    target = gpf.gpf_radiance_fwd(tidx, tf, queries, gpf.GPF_SUM, r_max=R_MAX)[0].clone()
    del tidx, tf
    grid, _ = autotune(field, queries, r_max=R_MAX, repeats=4)
    idx = make_index(field, queries, grid=grid, headroom=1.25)
    step = TrainStep(field, queries, target, idx, r_max=R_MAX, lr=LR)
    step.capture(warmup=1)                      # one real step, then the recording
    n = args.train_steps
    losses = torch.empty((n,), dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(n):
        step()
        losses[i].copy_(step.loss[0])
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / n
    st = idx.stats()
    if st["overflow"]:
        raise RuntimeError(f"pair buffer overflow: {st}")
    lh = losses.cpu().numpy().astype(float)
    marks = sorted({0, n // 4, n // 2, 3 * n // 4, n - 1})
    line = {
        "metric": "training-step hit-point queries/s (8 views, 1M Gaussians)",
        "value": n_active / (ms / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": n,
        "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{N_PHOTONS:,} Gaussians, 8 orbit views of 800x800, "
                               f"{n} Adam steps, CUDA graph",
                   "hit_points": int(qnp.m), "active_hit_points": n_active,
                   "l2": "inputs larger than L2",
                   "grid": {"query_cell": grid.cell_size * (1 << grid.query_level),
                            "max_span": grid.max_span, "coop_cells": grid.coop_cells,
                            "split_items": grid.split_items}},
        "loss": {str(i + 2): lh[i] for i in marks},   # step 1 ran before the capture
        "loss_ratio_last_first": lh[-1] / lh[0],
        "setup_s": {"generate": round(gen_s, 1)},
    }
    print(json.dumps(line), flush=True)


def run_bf16(args):
    """16-bit parameter storage: 4M Gaussians with an 8-bin spectrum in
    Morton order, 16 views of 1920x1080; the captured training step with
    float32 parameters, with GPF_BF16_MEAN32 and with GPF_BF16 storage (the
    16-bit forms update a float32 master and re-quantise it), and the
    relative difference of each 16-bit form's radiance from the float32
    form's on 4,096 random valid pixels (GPU outputs only)."""
    import torch
    import synth
    from synth import storage
    import paper_2512_12459_gb300 as gpf
    from paper_2512_12459_gb300.setup_index import make_index
    from paper_2512_12459_gb300.train import TrainStep

    torch.cuda.set_device(0)
    t0 = time.time()
    pos, flux = synth.caustic_photons(args.bf16_photons, seed=0, channels=8)
    fnp = synth.field_from_photons(pos, flux, seed=0)
    fnp = storage.permuted(fnp, storage.morton_order(fnp))
    tgt_np = synth.perturbed_copy(fnp, seed=1)
    qnp = synth.orbit_views(args.bf16_views, 1920, 1080)
    gen_s = time.time() - t0
    queries = gpf.Queries.from_numpy(qnp)
    n_active = int(qnp.valid.sum())
    tf = gpf.Field.from_numpy(tgt_np)
    tidx = make_index(tf, queries, query_cell=CELL)
    tidx.build(tf, queries)
    target, _ = gpf.gpf_radiance_fwd(tidx, tf, queries, gpf.GPF_SUM, r_max=R_MAX)
    target = target.clone()
    del tidx, tf
    torch.cuda.empty_cache()

    rng = np.random.default_rng(7)
    sel = torch.as_tensor(rng.choice(np.flatnonzero(qnp.valid.astype(bool)), 4096, replace=False),
                          device="cuda")
    results, first = {}, {}
    for name in ("f32", "bf16_mean32", "bf16"):
        master = gpf.Field.from_numpy(fnp)
        store = None if name == "f32" else master.quantized(mean32=(name == "bf16_mean32"))
        read = master if store is None else store
        idx = make_index(read, queries, query_cell=CELL, max_span=3, coop_cells=8, headroom=1.25)
        idx.build(read, queries)
        o, _ = gpf.gpf_radiance_fwd(idx, read, queries, gpf.GPF_SUM, r_max=R_MAX)
        first[name] = o[:, sel].double().cpu().numpy()
        del o
        step = TrainStep(master, queries, target, idx, r_max=R_MAX, lr=LR, store=store)
        step.capture(warmup=args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        pbytes = sum(t.numel() * t.element_size() for t in read.tensors())
        if store is not None:
            pbytes += store.anchor.numel() * 4
        results[name] = {"ms_per_step": ms, "queries_per_s": n_active / (ms / 1e3),
                         "param_bytes": pbytes}
        del step, idx, master, store, read
        torch.cuda.empty_cache()
    ref = first["f32"]
    for name in ("bf16_mean32", "bf16"):
        rel = np.abs(first[name] - ref) / np.maximum(np.abs(ref), 1e-30)
        pp = rel.max(axis=0)
        results[name]["rel_diff_vs_f32"] = {"median": float(np.median(pp)),
                                            "p99": float(np.percentile(pp, 99)),
                                            "max": float(pp.max())}
    line = {
        "metric": METRIC, "value": results["bf16_mean32"]["queries_per_s"], "unit": "queries/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": results["bf16_mean32"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 storage, f32 compute",
        "data": "synthetic",
        "config": {"workload": f"{fnp.n:,} Gaussians (8-bin spectrum, Morton order), "
                               f"{args.bf16_views} views of 1920x1080, CUDA graph",
                   "hit_points": int(qnp.m), "active_hit_points": n_active,
                   "l2": "inputs larger than L2"},
        "forms": results, "setup_s": {"generate": round(gen_s, 1)},
    }
    print(json.dumps(line), flush=True)


def run_kde(args):
    """The per-view photon density estimate (GPF_DISK_KDE) on the bench
    scene: the same 1M photons gathered within r = 0.02 at the 1024x1024
    view's hit points; index build + gather per step, L2 flushed between
    steps."""
    import torch
    import synth
    import paper_2512_12459_gb300 as gpf
    from paper_2512_12459_gb300.setup_index import autotune, make_index

    torch.cuda.set_device(0)
    pos, flux = synth.caustic_photons(N_PHOTONS, seed=0)
    qnp = synth.pinhole_hitpoints(EYE0, LOOK_AT, VIEW, VIEW)
    n_active = int(qnp.valid.sum())
    photons = gpf.photon_field(torch.as_tensor(pos.T.copy(), dtype=torch.float32, device="cuda"),
                               torch.as_tensor(flux.T.copy(), dtype=torch.float32, device="cuda"),
                               R_MAX)
    queries = gpf.Queries.from_numpy(qnp)
    # the dense caustic cores put up to ~10^5 photons in a tile's lists: tiles
    # are split over several work units while the grid is tuned
    grid, _ = autotune(photons, queries, mode=gpf.GPF_DISK_KDE, r_max=R_MAX, repeats=1,
                       max_spans=(3, 4, 6, 8), coop_options=(1, 2, 4, 8), backward=False,
                       split_options=(8192, 2048, 32768, 0))
    idx = make_index(photons, queries, grid=grid)
    out = torch.empty((3, queries.m), device="cuda")
    z = torch.empty((queries.m,), device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        idx.build(photons, queries)
        gpf.gpf_radiance_fwd(idx, photons, queries, gpf.GPF_DISK_KDE, r_max=R_MAX, out=out, z=z)
    torch.cuda.synchronize()
    marks = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        idx.build(photons, queries)
        ev[1].record()
        gpf.gpf_radiance_fwd(idx, photons, queries, gpf.GPF_DISK_KDE, r_max=R_MAX, out=out, z=z)
        ev[2].record()
        marks.append(ev)
    torch.cuda.synchronize()
    build_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in marks]))
    gather_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in marks]))
    gathered = float(z.sum().item())
    line = {
        "metric": "hit-point photon density estimates/sec (disk kernel, build + gather)",
        "value": n_active / ((build_ms + gather_ms) / 1e3), "unit": "queries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": build_ms + gather_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{N_PHOTONS:,} caustic photons, {VIEW}x{VIEW} view, r={R_MAX}",
                   "active_hit_points": n_active, "l2": "flushed between steps"},
        "gather_queries_per_s": n_active / (gather_ms / 1e3),
        "ms_breakdown": {"build": build_ms, "gather": gather_ms},
        "photons_gathered": gathered, "photons_per_hit_point": gathered / max(n_active, 1),
        "grid": {"query_cell": grid.cell_size * (1 << grid.query_level), "levels": grid.levels,
                 "max_span": grid.max_span, "coop_cells": grid.coop_cells,
                 "split_items": grid.split_items},
    }
    print(json.dumps(line), flush=True)


def run_scaling(args):
    """Table S1's experiment as throughput: the caustic scene's training step
    (build, forward, MSE, backward, Adam; autotuned grid) on the 1024x1024
    view for the paper's field sizes (10K-200K Gaussians) and this build's
    (0.5M-2M), L2 flushed between steps; one JSON object per size."""
    import torch
    import synth
    import paper_2512_12459_gb300 as gpf
    from paper_2512_12459_gb300.setup_index import autotune, make_index

    torch.cuda.set_device(0)
    qnp = synth.pinhole_hitpoints(EYE0, LOOK_AT, VIEW, VIEW)
    queries = gpf.Queries.from_numpy(qnp)
    n_active = int(qnp.valid.sum())
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = []
    for n in (10_000, 50_000, 100_000, 200_000, 500_000, 1_000_000, 2_000_000):
        pos, flux = synth.caustic_photons(n, seed=0)
        fnp = synth.field_from_photons(pos, flux, seed=0)
        tgt = gpf.Field.from_numpy(synth.perturbed_copy(fnp, seed=1))
        field = gpf.Field.from_numpy(fnp)
        ti = make_index(tgt, queries, query_cell=CELL)
        ti.build(tgt, queries)
        target = gpf.gpf_radiance_fwd(ti, tgt, queries, gpf.GPF_SUM, r_max=R_MAX)[0].clone()
        del ti
        grid, _ = autotune(field, queries, r_max=R_MAX, repeats=1)
        idx = make_index(field, queries, grid=grid, headroom=1.25)
        state = gpf.AdamState.zeros_like(field)
        grads = gpf.Field.zeros_like(field)
        out = torch.empty((3, queries.m), device="cuda")
        z = torch.empty((queries.m,), device="cuda")
        gout = torch.empty_like(out)

        def step(ev=None):
            if ev:
                ev[0].record()
            idx.build(field, queries)
            gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=R_MAX, out=out, z=z)
            if ev:
                ev[1].record()
            gpf.gpf_mse_loss_grad(out, target, queries.valid, grad=gout)
            gpf.gpf_radiance_bwd(idx, field, queries, gout, out, z, gpf.GPF_SUM, r_max=R_MAX,
                                 grads=grads)
            gpf.gpf_adam_step(field, grads, state, lr=LR)
            if ev:
                ev[2].record()

        for _ in range(args.warmup):
            step()
        marks = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            step(ev)
            marks.append(ev)
        torch.cuda.synchronize()
        fwd_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in marks]))
        step_ms = float(np.mean([e[0].elapsed_time(e[2]) for e in marks]))
        pairs = gpf.gpf_count_pairs(idx, field, queries)
        rows.append({"gaussians": n, "ms_per_step": step_ms, "queries_per_s": n_active / step_ms * 1e3,
                     "build_fwd_ms": fwd_ms, "included_pairs_per_query": pairs["included"] / n_active})
        del idx, field, state, grads, target
        torch.cuda.empty_cache()
    # the paper's own query (ball r = 0.02 or the k_min nearest, normalised):
    # build + forward against the field size (Table S1) and against k_min at
    # 100K Gaussians (Table S2)
    hyb_rows, k_rows = [], []

    def hybrid_ms(n, k_min):
        pos, flux = synth.caustic_photons(n, seed=0)
        field = gpf.Field.from_numpy(synth.field_from_photons(pos, flux, seed=0))
        idx = make_index(field, queries, query_cell=CELL, ball_radius=R_MAX)
        out = torch.empty((3, queries.m), device="cuda")
        z = torch.empty((queries.m,), device="cuda")
        times = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            idx.build(field, queries)
            gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_NORMALIZED, r_max=R_MAX, out=out,
                                 z=z, neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=R_MAX,
                                 k_min=k_min)
            e1.record()
            e1.synchronize()
            if i >= args.warmup:
                times.append(e0.elapsed_time(e1))
        del idx, field
        torch.cuda.empty_cache()
        return float(np.mean(times))

    def hybrid_step_ms(n, k_min):
        # the paper's training step through its own neighbourhood: build,
        # hybrid forward, MSE, hybrid backward (the selected pairs sorted by
        # Gaussian), Adam; the pair room from a trial step
        pos, flux = synth.caustic_photons(n, seed=0)
        fnp = synth.field_from_photons(pos, flux, seed=0)
        field = gpf.Field.from_numpy(fnp)
        tgt = gpf.Field.from_numpy(synth.perturbed_copy(fnp, seed=1))
        kw = dict(neighbourhood=gpf.GPF_NB_BALL_KNN, ball_r=R_MAX, k_min=k_min)
        ti = make_index(tgt, queries, query_cell=CELL, ball_radius=R_MAX)
        ti.build(tgt, queries)
        target = gpf.gpf_radiance_fwd(ti, tgt, queries, gpf.GPF_NORMALIZED, r_max=R_MAX,
                                      **kw)[0].clone()
        del ti
        state = gpf.AdamState.zeros_like(field)
        grads = gpf.Field.zeros_like(field)
        out = torch.empty((3, queries.m), device="cuda")
        z = torch.empty((queries.m,), device="cuda")
        gout = torch.empty_like(out)
        cap = 64 * queries.m
        for _ in range(3):
            idx = make_index(field, queries, query_cell=CELL, ball_radius=R_MAX, max_nb_pairs=cap)

            def step():
                idx.build(field, queries)
                gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_NORMALIZED, r_max=R_MAX,
                                     out=out, z=z, **kw)
                gpf.gpf_mse_loss_grad(out, target, queries.valid, grad=gout)
                gpf.gpf_radiance_bwd(idx, field, queries, gout, out, z, gpf.GPF_NORMALIZED,
                                     r_max=R_MAX, grads=grads, **kw)
                gpf.gpf_adam_step(field, grads, state, lr=LR, guard=idx)

            step()
            st = idx.stats()
            if not st["overflow"]:
                break
            cap = int(st["n_nb_pairs"] * 1.1) + 1024
            del idx
            torch.cuda.empty_cache()
        times = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            e1.synchronize()
            if i >= args.warmup:
                times.append(e0.elapsed_time(e1))
        pairs = idx.stats()["n_nb_pairs"]
        del idx, field, state, grads, target
        torch.cuda.empty_cache()
        return float(np.mean(times)), pairs

    step_rows = []
    for n in (10_000, 100_000):
        ms, pairs = hybrid_step_ms(n, 3)
        step_rows.append({"gaussians": n, "k_min": 3, "ms_per_step": ms, "selected_pairs": pairs,
                          "queries_per_s": n_active / ms * 1e3})
    for n in (10_000, 50_000, 100_000, 200_000):
        ms = hybrid_ms(n, 3)
        hyb_rows.append({"gaussians": n, "k_min": 3, "build_fwd_ms": ms,
                         "queries_per_s": n_active / ms * 1e3})
    for k in (1, 3, 5, 10):
        ms = hybrid_ms(100_000, k)
        k_rows.append({"gaussians": 100_000, "k_min": k, "build_fwd_ms": ms,
                       "queries_per_s": n_active / ms * 1e3})
    line = {"metric": "training step time vs number of Gaussians (Table S1 replay)",
            "value": rows[-1]["queries_per_s"], "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"caustic scene, {VIEW}x{VIEW} view, r={R_MAX}",
                       "active_hit_points": n_active, "l2": "flushed between steps"},
            "rows": rows,
            "hybrid_query_rows": hyb_rows, "hybrid_k_rows": k_rows,
            "hybrid_training_step_rows": step_rows,
            "paper_table_s1_s": {"10000": 7.230, "50000": 12.70, "100000": 16.37, "200000": 24.35},
            "paper_table_s2_s": {"1": 16.21, "3": 16.37, "5": 16.48, "10": 16.34}}
    print(json.dumps(line), flush=True)


def main():
    global N_PHOTONS, VIEW, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpf", choices=["gpf", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--photons", type=int, default=N_PHOTONS,
                    help="Gaussians (smaller cases are for profiling only)")
    ap.add_argument("--view", type=int, default=VIEW, help="view side in pixels")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batched", "bf16", "kde", "scaling", "train"],
                    help="single: the 1M-Gaussian 1024x1024 step (default line); batched: "
                         "64 uneven views over 2M Gaussians, graph replay vs per-view launches")
    ap.add_argument("--batched-views", type=int, default=64)
    ap.add_argument("--train-steps", type=int, default=200,
                    help="train workload: Adam steps timed")
    ap.add_argument("--batched-photons", type=int, default=2_000_000)
    ap.add_argument("--bf16-photons", type=int, default=4_000_000)
    ap.add_argument("--bf16-views", type=int, default=16)
    ap.add_argument("--grid", default=None, metavar="QUERY_CELL,MAX_SPAN,COOP[,SPLIT]",
                    help="single workload: this grid instead of the autotuned one (the "
                         "profiling commands pin the grid the autotuner chose, so that every "
                         "run captures the same launches)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if (args.photons, args.view) != (N_PHOTONS, VIEW):
        N_PHOTONS, VIEW = args.photons, args.view
        WORKLOAD = (f"caustic floor+sphere scene, {N_PHOTONS:,} Gaussians, {VIEW}x{VIEW} view, "
                    "3-sigma grid, r=0.02 (reduced profiling case)")

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "bf16":
        run_bf16(args)
        return
    if args.workload == "kde":
        run_kde(args)
        return
    if args.workload == "scaling":
        run_scaling(args)
        return
    if args.workload == "train":
        run_train(args)
        return

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import paper_2512_12459_gb300 as gpf
    from paper_2512_12459_gb300 import sharding
    from paper_2512_12459_gb300.setup_index import autotune, make_index

    fnp, tgt_np, qnp = make_inputs(rank)
    # the oracle's process pool starts now (spawned: it shares nothing with
    # this process's CUDA context) and is used after the timed region
    pool = OraclePool(fnp) if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    field = gpf.Field.from_numpy(fnp)
    field0 = gpf.Field(*(t.clone() for t in field.tensors()))   # before any Adam step
    queries = gpf.Queries.from_numpy(qnp)
    tgt_field = gpf.Field.from_numpy(tgt_np)
    n_active = int(qnp.valid.sum())
    # every rank's MSE is normalised by its own valid points; the gradients
    # are combined with weights n_active / n_total (the MSE over all views)
    n_total = sharding.global_count(n_active, device="cuda") if world > 1 else n_active

    # target radiance: the perturbed field rendered through the same path (outside timing)
    tidx = make_index(tgt_field, queries, query_cell=CELL, cutoff_sigma=CUTOFF)
    tidx.build(tgt_field, queries)
    target, _ = gpf.gpf_radiance_fwd(tidx, tgt_field, queries, gpf.GPF_SUM, r_max=R_MAX)
    target = target.clone()
    del tidx

    # grid geometry and forward tile shape chosen by timing candidates on this
    # scene (outside the timed region); headroom for the pairs to grow as
    # Adam moves the Gaussians
    if args.grid:
        parts = args.grid.split(",")
        qc, span, coop = parts[:3]
        idx = make_index(field, queries, cutoff_sigma=CUTOFF, headroom=1.25,
                         query_cell=float(qc), max_span=int(span), coop_cells=int(coop),
                         split_items=int(parts[3]) if len(parts) > 3 else 0)
    else:
        tuned, _ = autotune(field, queries, cutoff_sigma=CUTOFF, r_max=R_MAX, repeats=4)
        idx = make_index(field, queries, grid=tuned, headroom=1.25)
    state = gpf.AdamState.zeros_like(field)
    grads = gpf.Field(*(torch.empty_like(t) for t in field.tensors()))
    out = torch.empty((3, queries.m), device="cuda")
    z = torch.empty((queries.m,), device="cuda")
    gout = torch.empty_like(out)
    loss = torch.empty((1,), device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    ev = {k: [] for k in ("step", "build", "fwd", "loss", "bwd", "adam")}

    def step(timed: bool, q=queries, tgt=target):
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(10)] if timed else None
        if timed:
            # the library records marks[6:8] / marks[8:10] around the forward
            # and backward pair-loop kernels themselves
            idx.set_timing_events(fwd=(marks[6], marks[7]), bwd=(marks[8], marks[9]))
            marks[0].record(stream)
        idx.build(field, q)
        if timed:
            marks[1].record(stream)
        gpf.gpf_radiance_fwd(idx, field, q, gpf.GPF_SUM, r_max=R_MAX, out=out, z=z)
        if timed:
            marks[2].record(stream)
        gpf.gpf_mse_loss_grad(out, tgt, q.valid, loss=loss, grad=gout)
        if timed:
            marks[3].record(stream)
        gpf.gpf_radiance_bwd(idx, field, q, gout, out, z, gpf.GPF_SUM, r_max=R_MAX,
                             grads=grads)
        if world > 1:
            sharding.allreduce_gradients(grads.tensors(), n_active, n_total)
        if timed:
            marks[4].record(stream)
        gpf.gpf_adam_step(field, grads, state, lr=LR)
        if timed:
            marks[5].record(stream)
        return marks

    idx.set_timing_events()
    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    st = idx.stats()
    if st["overflow"]:
        raise RuntimeError(f"pair buffer overflow in warm-up: {st}")
    launches0 = gpf.gpf_launch_count()

    sampler = ClockSampler(local_rank)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    all_marks = []
    for _ in range(args.steps):
        flush.fill_(1.0)          # evict L2 between timed steps (not timed)
        all_marks.append(step(True))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    idx.set_timing_events()
    launches = gpf.gpf_launch_count() - launches0

    per = {k: [] for k in ("build", "fwd", "loss", "bwd", "adam", "step")}
    for mk in all_marks:
        names = ("build", "fwd", "loss", "bwd", "adam")
        for i, nm in enumerate(names):
            per[nm].append(mk[i].elapsed_time(mk[i + 1]))
        per["step"].append(mk[0].elapsed_time(mk[5]))
    ms = {k: float(np.mean(v)) for k, v in per.items()}
    kernel_ms = {"fwd_kernel": float(np.mean([mk[6].elapsed_time(mk[7]) for mk in all_marks])),
                 "bwd_grid_kernel": float(np.mean([mk[8].elapsed_time(mk[9]) for mk in all_marks]))}
    step_ms = sharding.max_over_ranks(ms["step"], device="cuda")
    total_q = float(n_total)
    value = total_q / (step_ms / 1000.0)

    # pair counts for the roofline (outside timing)
    pairs = gpf.gpf_count_pairs(idx, field, queries)

    # end to end through the public API with host buffers: every step copies
    # its hit points and target from pinned host memory and reads its loss
    # back. The copies run on their own stream into two alternating input
    # sets, so that step i + 1's inputs arrive while step i computes (a set
    # is overwritten only after the step that used it is done).
    host = {k: torch.as_tensor(v).pin_memory() for k, v in
            (("x", qnp.x), ("n", qnp.n), ("wo", qnp.wo), ("valid", qnp.valid))}
    host["target"] = target.cpu().pin_memory()
    loss_host = torch.empty((2,), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = 4
    sets = [(gpf.Queries(torch.empty_like(queries.x), torch.empty_like(queries.normal),
                         torch.empty_like(queries.wo), None, torch.empty_like(queries.valid)),
             torch.empty_like(target)) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]

    def issue_copy(i):
        qs, ts = sets[i % 2]
        with torch.cuda.stream(copy_stream):
            if i >= 2:
                copy_stream.wait_event(used[i % 2])
            qs.x.copy_(host["x"], non_blocking=True)
            qs.normal.copy_(host["n"], non_blocking=True)
            qs.wo.copy_(host["wo"], non_blocking=True)
            qs.valid.copy_(host["valid"], non_blocking=True)
            ts.copy_(host["target"], non_blocking=True)
            copied[i % 2].record(copy_stream)

    def run_e2e(n_steps):
        issue_copy(0)
        for i in range(n_steps):
            if i + 1 < n_steps:
                issue_copy(i + 1)
            stream.wait_event(copied[i % 2])
            qs, ts = sets[i % 2]
            step(False, qs, ts)
            loss_host[i % 2].copy_(loss[0], non_blocking=True)
            used[i % 2].record(stream)

    run_e2e(args.warmup)
    torch.cuda.synchronize()
    flush.fill_(1.0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy_stream.wait_stream(stream)
    run_e2e(args.steps)
    e1.record(stream)
    e1.synchronize()
    e2e_times = [e0.elapsed_time(e1) / args.steps]
    e2e_ms = sharding.max_over_ranks(float(np.mean(e2e_times)), device="cuda")

    peaks, peaks_src = measured_peaks()
    smax = float(peaks.get("sm_max_mhz", 2070.0))
    nominal_fp32 = fp32_peak_tflops(smax)
    # the pipes the pair loops use, measured on this GPU (after the timed region)
    fma = gpf.gpf_measure_alu_peak(gpf.GPF_PEAK_FP32_FMA)
    ex2 = gpf.gpf_measure_alu_peak(gpf.GPF_PEAK_EX2)
    fp32_peak = fma["per_second"] / 1e12
    ex2_peak = ex2["per_second"] / 1e12
    alu_peaks = {"fp32_fma_tflops": fp32_peak, "ex2_tops": ex2_peak,
                 "fp32_nominal_tflops": nominal_fp32,
                 "how": "gpf_measure_alu_peak: 8 x 256 threads per SM, 8 independent chains "
                        "per thread, CUDA events"}
    C = fnp.channels
    roof = None
    extra = {}
    if pairs is not None:
        inc = pairs["included"]
        fwd_flops = inc * (25 + 2 * C)       # per included pair, FMA = 2 flops
        bwd_flops = inc * (55 + 4 * C)
        fwd_ach = fwd_flops / (kernel_ms["fwd_kernel"] / 1e3) / 1e12
        bwd_ach = bwd_flops / (kernel_ms["bwd_grid_kernel"] / 1e3) / 1e12
        dom = "bwd_grid_kernel" if kernel_ms["bwd_grid_kernel"] >= kernel_ms["fwd_kernel"] \
            else "fwd_kernel"
        ach = bwd_ach if dom == "bwd_grid_kernel" else fwd_ach
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": ach / fp32_peak, "traffic": profiled_traffic(dom),
                "peak_source": "measured FP32 FMA rate of this GPU (gpf_measure_alu_peak); "
                               f"nominal 152 SMs x 128 lanes x 2 x {smax:.0f} MHz = "
                               f"{nominal_fp32:.1f}",
                "duration_ms": kernel_ms[dom]}
        # one ex2 per included pair in either pair loop
        extra = {"included_pairs": inc, "candidate_pairs": pairs["candidates"],
                 "fwd_alu_frac": fwd_ach / fp32_peak, "bwd_alu_frac": bwd_ach / fp32_peak,
                 "fwd_sfu_frac": inc / (kernel_ms["fwd_kernel"] / 1e3) / 1e12 / ex2_peak,
                 "bwd_sfu_frac": inc / (kernel_ms["bwd_grid_kernel"] / 1e3) / 1e12 / ex2_peak}

    cpu, err = None, None
    if pool is not None:
        tgt_out = target.cpu().numpy().astype(np.float64)
        rate, done, dt, results = pool.run(qnp, lambda sel: tgt_out[:, sel],
                                           budget_s=args.cpu_budget)
        pool.close()
        cpu = {"value": rate, "unit": "queries/s", "cores": pool.cores, "kind": "oracle",
               "sample": f"{done} random valid hit points of the same view, fwd+bwd each over all "
                         f"1,000,000 Gaussians, {dt:.1f} s (numpy float64, one process per "
                         "core)"}
        # the error of the GPU forward at the same points (the field before
        # the steps above, through a fresh build of the same index)
        idx.build(field0, queries)
        out0, _ = gpf.gpf_radiance_fwd(idx, field0, queries, gpf.GPF_SUM, r_max=R_MAX)
        err = error_vs_oracle(out0.cpu().numpy().astype(np.float64), results)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": int(total_q), "seq_len": None,
                       "parallelism": f"dp{world}", "hit_points_per_gpu": n_active,
                       "gaussians": fnp.n, "l2": "flushed between steps",
                       "grid": {"query_cell": idx.grid.cell_size * (1 << idx.grid.query_level),
                                "levels": idx.grid.levels, "finest_cell": idx.grid.cell_size,
                                "max_span": idx.grid.max_span,
                                "coop_cells": idx.grid.coop_cells,
                                "split_items": idx.grid.split_items,
                                "autotuned": not args.grid}},
            "fwd_queries_per_s": n_active / (ms["fwd"] / 1e3),
            "fwd_bwd_queries_per_s": n_active / ((ms["fwd"] + ms["bwd"] + ms["loss"]) / 1e3),
            "ms_breakdown": {k: v for k, v in ms.items() if k != "step"},
            "kernel_ms": kernel_ms,
            "roofline": roof,
            "alu_peaks": alu_peaks,
            "cpu_baseline": cpu,
            "error_vs_oracle": err,
            "e2e": {"value": total_q / (e2e_ms / 1e3), "unit": "queries/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms,
                    "copies": "own stream, two alternating input sets (step i+1's inputs "
                              "arrive while step i runs)"},
            "gpu_launches": launches,
            "clocks": clocks,
            "index": {"n_pairs": st["n_pairs"], "max_pairs": idx.grid.max_pairs},
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
