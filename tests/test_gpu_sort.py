"""The index build's radix sort through the C ABI (gpf_sort_pairs): stable
order against numpy's stable argsort on sizes around the 3072-key tile and
up to millions of keys, and the bounded wait of its single-pass kernel
(gpf_test_sort_wait_timeout: a look-back whose predecessor never publishes
gives up, reports GPF_ERR_TIMEOUT and leaves the context usable)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12459_gb300 as g
    return g


def _keys(kind, n, bits, rng):
    hi = 1 << bits
    if kind == "uniform":
        k = rng.integers(0, hi, n, dtype=np.uint64)
    elif kind == "few":                      # long runs of equal keys
        k = rng.integers(0, 4, n, dtype=np.uint64) * (hi // 4)
    elif kind == "sorted":
        k = np.sort(rng.integers(0, hi, n, dtype=np.uint64))
    elif kind == "reversed":
        k = np.sort(rng.integers(0, hi, n, dtype=np.uint64))[::-1]
    else:                                    # all equal
        k = np.full(n, hi - 1, dtype=np.uint64)
    return k.astype(np.uint32)


def _run(gpf, keys_u32, bits):
    import torch
    n = keys_u32.size
    vals = np.arange(n, dtype=np.uint32)[::-1].copy()       # distinct: exposes instability
    tk = torch.from_numpy(keys_u32.view(np.int32)).cuda()
    tv = torch.from_numpy(vals.view(np.int32)).cuda()
    ok, ov = gpf.gpf_sort_pairs(tk, tv, bits)
    order = np.argsort(keys_u32, kind="stable")
    got_k = ok.cpu().numpy().view(np.uint32)
    got_v = ov.cpu().numpy().view(np.uint32)
    assert np.array_equal(got_k, keys_u32[order])
    assert np.array_equal(got_v, vals[order])


@pytest.mark.parametrize("n", [1, 31, 2048, 3071, 3072, 3073, 9215, 100_003])
@pytest.mark.parametrize("bits", [8, 13, 24, 32])
def test_sort_small_sizes_every_pass_count(gpf, n, bits):
    rng = np.random.default_rng(n * 100 + bits)
    _run(gpf, _keys("uniform", n, bits, rng), bits)


@pytest.mark.parametrize("kind", ["uniform", "few", "sorted", "reversed", "equal"])
def test_sort_key_distributions(gpf, kind):
    rng = np.random.default_rng(7)
    _run(gpf, _keys(kind, 300_001, 24, rng), 24)


def test_sort_many_tiles(gpf):
    """5 M pairs: 1,628 tiles per pass, 3 passes (the entry sort's size)."""
    rng = np.random.default_rng(11)
    _run(gpf, _keys("uniform", 5_000_000, 24, rng), 24)


def test_sort_empty(gpf):
    import torch
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    k, v = gpf.gpf_sort_pairs(e, e.clone(), 24)
    assert k.numel() == 0 and v.numel() == 0


def test_sort_wait_gives_up_and_reports(gpf):
    import torch
    from paper_2512_12459_gb300 import _abi
    lib = gpf.load()
    st = lib.gpf_test_sort_wait_timeout(1 << 14, None)
    assert st == _abi.GPF_ERR_TIMEOUT
    assert b"gave up" in lib.gpf_last_error()
    # the context is still usable: a sort right after it is correct
    rng = np.random.default_rng(3)
    _run(gpf, _keys("uniform", 50_000, 24, rng), 24)
    torch.cuda.synchronize()
