"""The GPF_BF16 storage form on the host: rounding, the encoder's error
bounds, and the C ABI's validation of 16-bit fields (no GPU)."""

import ctypes

import numpy as np
import pytest

import synth
from synth import storage

torch = pytest.importorskip("torch")


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e-8, 65504.0, 1.0 + 2.0 ** -9,
                  1.0 + 2.0 ** -8 + 2.0 ** -20], dtype=np.float32)
    h = storage.f32_to_bf16(x)
    assert h[0] == 0x3F80                      # exact
    assert h[1] == 0x3F80                      # tie -> even
    assert h[2] == 0x3F82                      # tie -> even (up)
    assert h[6] == 0x3F80 and h[7] == 0x3F81   # below / above the tie
    # an independent implementation of the same rounding
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(h, ref)
    rng = np.random.default_rng(0)
    y = (rng.standard_normal(100000) * 10.0 ** rng.uniform(-6, 6, 100000)).astype(np.float32)
    ref = torch.from_numpy(y).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(storage.f32_to_bf16(y), ref)
    assert np.array_equal(storage.bf16_to_f32(ref), torch.from_numpy(ref.view(np.int16)).view(
        torch.bfloat16).float().numpy())


def test_encoder_error_bounds_follow_the_group_ranges():
    pos, flux = synth.caustic_photons(20000, seed=3)
    f0 = synth.field_from_photons(pos, flux, seed=3)
    f = storage.permuted(f0, storage.morton_order(f0))
    b = storage.encode(f)
    d = storage.decode(b)
    n = f.mean.shape[1]
    grp = np.arange(n) // storage.GROUP
    g = b.anchor.shape[0]
    assert b.anchor.shape == (g, 4) and g == (n + 15) // 16
    for k in range(3):
        col = f.mean[k].astype(np.float64)
        half = np.zeros(g)
        for j in range(g):
            s = col[j * 16:(j + 1) * 16]
            half[j] = 0.5 * (s.max() - s.min())
        err = np.abs(d.mean[k].astype(np.float64) - col)
        # bfloat16 keeps 8 significant bits: error <= 2^-8 |offset| plus the float32 sums
        assert np.all(err <= half[grp] * 2.0 ** -8 + 4 * 2.0 ** -24 * np.abs(col) + 1e-12)
    lerr = np.abs(d.logscale.astype(np.float64) - f.logscale)
    assert np.all(lerr <= 2.0 ** -8 * np.abs(f.logscale - b.anchor[grp, 3]) + 1e-6)
    assert np.all(np.abs(d.quat - f.quat) <= 2.0 ** -8 * np.abs(f.quat))
    assert np.all(np.abs(d.spectrum - f.spectrum) <= 2.0 ** -8 * np.abs(f.spectrum))
    # Morton order keeps groups compact: far smaller spans than storage order
    def med_span(ff):
        return np.median([np.ptp(ff.mean[:, j * 16:(j + 1) * 16], axis=1).max()
                          for j in range(g)])
    assert med_span(f) < med_span(f0) / 20


def _lib():
    from paper_2512_12459_gb300 import _abi
    import os
    if not os.path.exists(_abi.LIB_PATH):
        pytest.skip("libgpf.so not built")
    return _abi.load(), _abi


def test_bf16_fields_are_validated():
    lib, _abi = _lib()
    fake = 1 << 40
    cfg = _abi.gpf_grid_config((ctypes.c_float * 3)(0, 0, 0), 0.1, 4, 4, 0,
                               (ctypes.c_int32 * 3)(10, 10, 10), 16, 3, 3.0, 0, 0,
                               _abi.GPF_BF16, 0.0, 100, 200, 1000)
    h = ctypes.c_void_p()
    assert lib.gpf_index_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    sz = ctypes.c_size_t()
    lib.gpf_index_workspace_size(h, ctypes.byref(sz))
    q = _abi.gpf_queries(20, fake, fake, fake, None, None)
    f32 = _abi.gpf_field(10, 3, _abi.GPF_F32, fake, fake, fake, fake, None)
    assert lib.gpf_build_index(h, ctypes.byref(f32), ctypes.byref(q), fake, sz.value, None) == 1
    assert b"storage" in lib.gpf_last_error()
    bf = _abi.gpf_field(10, 3, _abi.GPF_BF16, fake + 2, fake, fake, fake, None)
    assert lib.gpf_build_index(h, ctypes.byref(bf), ctypes.byref(q), fake, sz.value, None) == 1
    assert b"anchor" in lib.gpf_last_error()
    bf.anchor = fake + 8
    assert lib.gpf_build_index(h, ctypes.byref(bf), ctypes.byref(q), fake, sz.value, None) == 1
    bf.mean = fake + 1
    bf.anchor = fake
    assert lib.gpf_build_index(h, ctypes.byref(bf), ctypes.byref(q), fake, sz.value, None) == 1
    assert b"2-byte" in lib.gpf_last_error()
    lib.gpf_index_destroy(h)
    # quantize: src float32, dst bfloat16, same sizes
    src = _abi.gpf_field(10, 3, _abi.GPF_F32, fake, fake, fake, fake, None)
    dst = _abi.gpf_field(10, 3, _abi.GPF_BF16, fake, fake, fake, fake, fake)
    assert lib.gpf_field_quantize(ctypes.byref(dst), ctypes.byref(dst), None) == 1
    assert lib.gpf_field_quantize(ctypes.byref(src), ctypes.byref(src), None) == 1
    dst.n = 11
    assert lib.gpf_field_quantize(ctypes.byref(src), ctypes.byref(dst), None) == 1
    dst.n, dst.anchor = 10, fake + 4
    assert lib.gpf_field_quantize(ctypes.byref(src), ctypes.byref(dst), None) == 1
    # Adam updates float32 masters only
    g = _abi.gpf_field_grad(fake, fake, fake, fake, 0, 0)
    hp = _abi.gpf_adam_hparams((ctypes.c_float * 4)(5e-4, 5e-4, 5e-4, 5e-4), 0.9, 0.999, 1e-8, 1,
                               None)
    assert lib.gpf_adam_step(ctypes.byref(dst), ctypes.byref(g), ctypes.byref(g), ctypes.byref(g),
                             ctypes.byref(hp), None) == 1


def test_bfloat16_spectra_cannot_hold_a_1e3_per_pixel_bound():
    """The bound behind the 16-bit storage reading: a pixel carried by one
    Gaussian has O = rho w Phi, so a bfloat16 spectrum's rounding error is the
    pixel's error. Round to nearest keeps it below 2^-8 / (1 + 2^-8), the
    value Phi = 1 + 2^-8 (a tie, rounded to even: 1) reaches it, and over
    Exp(1) spectra the largest errors come close to it, far above 1e-3; a
    float16 spectrum (10 stored bits) stays below 2^-11 < 1e-3."""
    bound = 2.0 ** -8 / (1.0 + 2.0 ** -8)
    phi = np.array([1.0 + 2.0 ** -8], dtype=np.float32)
    got = storage.bf16_to_f32(storage.f32_to_bf16(phi))
    assert got[0] == 1.0
    np.testing.assert_allclose(abs(float(phi[0]) - float(got[0])) / float(phi[0]), bound,
                               rtol=1e-12)
    rng = np.random.default_rng(7)
    x = rng.exponential(1.0, 1_000_000).astype(np.float32)
    x = x[x > 1e-30]
    rel = np.abs(storage.bf16_to_f32(storage.f32_to_bf16(x)).astype(np.float64) - x) / x
    assert rel.max() <= bound * (1 + 1e-12)
    assert rel.max() > 3.5e-3 and np.quantile(rel, 0.5) > 5e-4
    half = np.abs(x.astype(np.float16).astype(np.float64) - x) / x
    assert half[x > 6.2e-5].max() <= 2.0 ** -11
