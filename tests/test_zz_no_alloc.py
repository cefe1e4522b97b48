"""gpf_mse_loss_grad_noalloc: the loss entry point for callers that cannot give
the library device memory. It must produce what the workspace-taking
gpf_mse_loss_grad produces, call after call, although all its calls share one
fixed scratch array inside the library. This file is collected last."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12459_gb300 as gpf
    return torch, gpf, gpf.load()


def _case(torch, m, c, seed):
    rng = np.random.default_rng(seed)
    out = torch.as_tensor(rng.standard_normal((c, m)).astype(np.float32), device="cuda")
    tgt = torch.as_tensor(rng.standard_normal((c, m)).astype(np.float32), device="cuda")
    valid = torch.as_tensor((rng.uniform(size=m) < 0.8).astype(np.uint8), device="cuda")
    return out, tgt, valid


def _noalloc(torch, lib, out, tgt, valid):
    c, m = out.shape
    loss = torch.full((1,), float("nan"), device="cuda")
    grad = torch.full_like(out, float("nan"))
    st = lib.gpf_mse_loss_grad_noalloc(m, c, out.data_ptr(), tgt.data_ptr(),
                                       None if valid is None else valid.data_ptr(),
                                       loss.data_ptr(), grad.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.gpf_last_error()
    return loss, grad


def test_noalloc_loss_matches_the_workspace_entry_point(env):
    torch, gpf, lib = env
    # two calls in a row (the second on a smaller problem, so stale partial
    # sums of the first would show), then the first problem again
    for m, c, seed in ((300001, 3, 1), (9000, 8, 2), (300001, 3, 1)):
        out, tgt, valid = _case(torch, m, c, seed)
        ref_loss, ref_grad = gpf.gpf_mse_loss_grad(out, tgt, valid)
        loss, grad = _noalloc(torch, lib, out, tgt, valid)
        torch.cuda.synchronize()
        # the same kernels in the same order: equal bit for bit, so a stale
        # partial sum left by the previous (larger) call would show
        np.testing.assert_array_equal(loss.cpu().numpy(), ref_loss.cpu().numpy())
        np.testing.assert_array_equal(grad.cpu().numpy(), ref_grad.cpu().numpy())
    # no valid mask, and an empty problem
    out, tgt, _ = _case(torch, 5000, 2, 3)
    ref_loss, ref_grad = gpf.gpf_mse_loss_grad(out, tgt, None)
    loss, grad = _noalloc(torch, lib, out, tgt, None)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(loss.cpu().numpy(), ref_loss.cpu().numpy())
    np.testing.assert_array_equal(grad.cpu().numpy(), ref_grad.cpu().numpy())
    e = torch.empty((3, 0), device="cuda")
    loss, _ = _noalloc(torch, lib, e, e, None)
    assert loss.item() == 0.0


def test_noalloc_refuses_sizes_beyond_its_array(env):
    torch, gpf, lib = env
    m = (1 << 26) + 1
    st = lib.gpf_mse_loss_grad_noalloc(m, 3, 1 << 40, 1 << 40, None, 1 << 40, 1 << 40, None)
    assert st == 1
    assert b"GPF_NOALLOC_MAX_POINTS" in lib.gpf_last_error()
