"""Failure detection without a GPU fault: an index build that cannot be used
(a pair buffer far too small for the scene, or a non-finite input) sets a
device flag; every later kernel that reads the index leaves its outputs
untouched, an Adam step guarded by the index is cancelled on the device, the
flags reach the host through gpf_index_flags_async without a synchronisation,
and gpf_index_stats reports the matching status. Nothing here waits on the
device beyond ordinary stream order."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12459_gb300 as g
    return g


def _snapshot(tensors):
    return [t.detach().clone() for t in tensors]


def _same(a, b):
    import torch
    return all(torch.equal(x, y) for x, y in zip(a, b))


def test_overflowed_build_cancels_a_captured_step(gpf):
    """A captured training step whose index overflows its pair buffer on every
    replay changes nothing: parameters, Adam moments, the device step counter,
    gradients and radiance stay bitwise as they were, and the step reports
    GPF_FLAG_CAPACITY through pinned host memory."""
    import torch
    from paper_2512_12459_gb300 import _abi
    from paper_2512_12459_gb300.setup_index import make_index
    from paper_2512_12459_gb300.train import TrainStep
    fnp, qnp = synth.config1_random(seed=40, n=2000, m=8000 + 3)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.1, max_pairs=64)     # far too small
    target = torch.rand((3, queries.m), device="cuda")
    step = TrainStep(field, queries, target, idx, r_max=0.05)
    # non-trivial moments and sentinels in every output, so that "untouched" means something
    g = torch.Generator(device="cuda").manual_seed(0)
    for t in step.state.m.tensors() + step.state.v.tensors():
        t.uniform_(0.1, 1.0, generator=g)
    for t in step.grads.tensors():
        t.fill_(7.0)
    step.out.fill_(5.0)
    step.z.fill_(3.0)
    step.state.step_counter.fill_(11)
    before = _snapshot(field.tensors() + step.state.m.tensors() + step.state.v.tensors() +
                       step.grads.tensors() + [step.out, step.z, step.state.step_counter])
    step.capture(warmup=1)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    after = field.tensors() + step.state.m.tensors() + step.state.v.tensors() + \
        step.grads.tensors() + [step.out, step.z, step.state.step_counter]
    assert _same(before, after)
    assert step.last_flags() == _abi.GPF_FLAG_CAPACITY
    st = idx.stats()
    assert st["overflow"] and st["flags"] == _abi.GPF_FLAG_CAPACITY and st["n_pairs"] > 64
    with pytest.raises(gpf.GPFError) as e:
        idx.stats(raise_on_flags=True)
    assert e.value.status == _abi.GPF_ERR_CAPACITY


def test_usable_build_reports_no_flags_and_steps(gpf):
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    from paper_2512_12459_gb300.train import TrainStep
    fnp, qnp = synth.config1_random(seed=41, n=2000, m=8000)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.1)
    step = TrainStep(field, queries, torch.rand((3, queries.m), device="cuda"), idx, r_max=0.05)
    before = _snapshot(field.tensors())
    step.capture(warmup=1)
    step()
    torch.cuda.synchronize()
    assert step.last_flags() == 0
    assert step.updates() == 2
    assert not _same(before, field.tensors())
    assert idx.stats()["flags"] == 0


@pytest.mark.parametrize("where", ["mean", "logscale", "spectrum", "hit_point"])
def test_non_finite_input_is_flagged_and_outputs_untouched(gpf, where):
    import torch
    from paper_2512_12459_gb300 import _abi
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp = synth.config1_random(seed=42, n=1500, m=5000)
    field, queries = gpf.Field.from_numpy(fnp), gpf.Queries.from_numpy(qnp)
    idx = make_index(field, queries, query_cell=0.1)
    if where == "hit_point":
        act = np.flatnonzero(np.sum(qnp.n * qnp.wo, axis=0) > 0)
        queries.x[1, int(act[7])] = float("nan")
    else:
        getattr(field, where)[0, 123] = float("nan")
    idx.build(field, queries)
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    idx.flags_async(flags)
    out = torch.full((3, queries.m), 5.0, device="cuda")
    z = torch.full((queries.m,), 3.0, device="cuda")
    gpf.gpf_radiance_fwd(idx, field, queries, gpf.GPF_SUM, r_max=0.05, out=out, z=z)
    grads = gpf.Field(*(torch.full_like(t, 7.0) for t in field.tensors()))
    gpf.gpf_radiance_bwd(idx, field, queries, torch.ones_like(out), r_max=0.05, grads=grads)
    torch.cuda.synchronize()
    assert int(flags.item()) == _abi.GPF_FLAG_NONFINITE
    assert torch.all(out == 5.0) and torch.all(z == 3.0)
    assert all(torch.all(t == 7.0) for t in grads.tensors())
    st = idx.stats()
    assert st["flags"] == _abi.GPF_FLAG_NONFINITE and not st["overflow"]
    with pytest.raises(gpf.GPFError) as e:
        idx.stats(raise_on_flags=True)
    assert e.value.status == _abi.GPF_ERR_NONFINITE


def test_backward_without_hit_points_writes_zeros(gpf):
    """No hit points: every gradient is zero (written by the epilogue), and
    accumulate=True leaves the existing values."""
    import torch
    from paper_2512_12459_gb300.setup_index import make_index
    fnp, qnp = synth.config1_random(seed=43, n=300, m=10)
    field = gpf.Field.from_numpy(fnp)
    empty = gpf.Queries(*(torch.empty((3, 0), device="cuda") for _ in range(3)))
    idx = make_index(field, empty, query_cell=0.1, max_pairs=1024)
    idx.build(field, empty)
    grads = gpf.Field(*(torch.full_like(t, 7.0) for t in field.tensors()))
    g0 = torch.empty((3, 0), device="cuda")
    gpf.gpf_radiance_bwd(idx, field, empty, g0, r_max=0.05, grads=grads, accumulate=True)
    torch.cuda.synchronize()
    assert all(torch.all(t == 7.0) for t in grads.tensors())
    gpf.gpf_radiance_bwd(idx, field, empty, g0, r_max=0.05, grads=grads)
    torch.cuda.synchronize()
    assert all(torch.all(t == 0.0) for t in grads.tensors())


def test_measured_alu_peaks_are_plausible(gpf):
    """The roofline denominators the benchmark reports: the FP32 FMA rate
    within what 152 SMs x 128 lanes x 2 flops can give at 1.0-2.1 GHz, and
    the ex2 rate between 8 and 64 results per SM per clock at those clocks."""
    fma = gpf.gpf_measure_alu_peak(gpf.GPF_PEAK_FP32_FMA, iters=2048)
    ex2 = gpf.gpf_measure_alu_peak(gpf.GPF_PEAK_EX2, iters=512)
    lanes = 152 * 128 * 2
    assert lanes * 1.0e9 < fma["per_second"] < lanes * 2.1e9, fma
    assert 152 * 8 * 1.0e9 < ex2["per_second"] < 152 * 64 * 2.1e9, ex2
    print(f"FP32 FMA {fma['per_second'] / 1e12:.1f} TFLOP/s, ex2 {ex2['per_second'] / 1e12:.2f} T/s")
