"""CPU-only checks of the C ABI: the library loads, exports every symbol that
include/gpf.h declares, and validates arguments on the host (no GPU call)."""

import ctypes
import math
import os
import re

import numpy as np
import pytest

from golden_util import load_constants


@pytest.fixture(scope="module")
def lib(root_dir):
    from paper_2512_12459_gb300 import _abi
    if not os.path.exists(_abi.LIB_PATH):
        from paper_2512_12459_gb300.build import build
        build()
    return _abi.load()


def _declared(root_dir):
    with open(os.path.join(root_dir, "include", "gpf.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gpf_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib, root_dir):
    from paper_2512_12459_gb300 import _abi
    names = _declared(root_dir)
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, f"binding lacks {name}"
    assert set(_abi.SIGNATURES) == set(names)


def test_version_and_status_strings(lib):
    assert b"sm_103a" in lib.gpf_version()
    for s, name in [(0, b"GPF_OK"), (1, b"GPF_ERR_INVALID_ARG"), (4, b"GPF_ERR_CAPACITY"),
                    (6, b"GPF_ERR_MISMATCH"), (7, b"GPF_ERR_TIMEOUT"),
                    (8, b"GPF_ERR_NONFINITE")]:
        assert lib.gpf_status_string(s) == name
    assert lib.gpf_status_string(99) == b"GPF_ERR_UNKNOWN"


def _cfg(**kw):
    from paper_2512_12459_gb300 import _abi
    c = _abi.gpf_grid_config((ctypes.c_float * 3)(0, 0, 0), 0.1, 4, 4, 0,
                             (ctypes.c_int32 * 3)(10, 10, 10), 16, 3, 3.0, 0, 0, 0, 0.0, 100, 200, 1000)
    for k, v in kw.items():
        if k == "dims":
            c.dims = (ctypes.c_int32 * 3)(*v)
        else:
            setattr(c, k, v)
    return c


@pytest.mark.parametrize("bad", [dict(cell_size=0.0), dict(cell_size=math.nan),
                                 dict(dims=(0, 10, 10)), dict(dims=(10, 2000, 10)),
                                 dict(channels=0), dict(channels=9), dict(cutoff_sigma=-1.0),
                                 dict(brute_force=2), dict(max_pairs=-5),
                                 dict(dims=(1024, 1024, 1024)), dict(levels=0), dict(levels=17),
                                 dict(max_span=0), dict(hash_bits=7), dict(hash_bits=29),
                                 dict(query_level=16), dict(query_level=11, dims=(1024, 4, 4)),
                                 dict(coop_cells=-1), dict(coop_cells=9), dict(field_storage=3),
                                 dict(ball_radius=-1.0), dict(ball_radius=math.inf),
                                 dict(max_pairs=1 << 30), dict(max_queries=1 << 30),
                                 dict(max_gaussians=1 << 30), dict(tile_order=-1),
                                 dict(tile_order=3), dict(tile_order=1),
                                 dict(tile_order=2, query_level=1)])
def test_index_create_rejects_bad_configs(lib, bad):
    h = ctypes.c_void_p()
    cfg = _cfg(**bad)
    assert lib.gpf_index_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert h.value is None
    assert len(lib.gpf_last_error()) > 0


def test_workspace_grows_with_capacity(lib):
    sizes = []
    for n in (100, 10000):
        h = ctypes.c_void_p()
        cfg = _cfg(max_gaussians=n, max_queries=n, max_pairs=8 * n)
        assert lib.gpf_index_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
        sz = ctypes.c_size_t()
        assert lib.gpf_index_workspace_size(h, ctypes.byref(sz)) == 0
        sizes.append(sz.value)
        lib.gpf_index_destroy(h)
    assert sizes[1] > sizes[0] > 0 and sizes[0] % 256 == 0


def test_host_validation_before_any_launch(lib):
    from paper_2512_12459_gb300 import _abi
    h = ctypes.c_void_p()
    cfg = _cfg()
    assert lib.gpf_index_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    sz = ctypes.c_size_t()
    lib.gpf_index_workspace_size(h, ctypes.byref(sz))
    fake = 1 << 40          # never dereferenced: validation fails first
    f = _abi.gpf_field(10, 3, 0, fake, fake, fake, fake)
    q = _abi.gpf_queries(20, fake, fake, fake, None, None)
    # no workspace
    assert lib.gpf_build_index(h, ctypes.byref(f), ctypes.byref(q), None, 0, None) == 1
    # workspace too small
    assert lib.gpf_build_index(h, ctypes.byref(f), ctypes.byref(q), fake, sz.value - 1,
                               None) == 3
    # misaligned workspace
    assert lib.gpf_build_index(h, ctypes.byref(f), ctypes.byref(q), fake + 4, sz.value,
                               None) == 1
    # too many Gaussians / hit points, wrong channel count, NULL arrays
    f.n = 101
    assert lib.gpf_build_index(h, ctypes.byref(f), ctypes.byref(q), fake, sz.value, None) == 1
    f.n, f.channels = 10, 4
    assert lib.gpf_build_index(h, ctypes.byref(f), ctypes.byref(q), fake, sz.value, None) == 1
    f.channels, f.mean = 3, None
    assert lib.gpf_build_index(h, ctypes.byref(f), ctypes.byref(q), fake, sz.value, None) == 1
    assert b"field.mean" in lib.gpf_last_error()
    f.mean = fake
    q.m = 201
    assert lib.gpf_build_index(h, ctypes.byref(f), ctypes.byref(q), fake, sz.value, None) == 1
    q.m = 20
    # forward before any build, and with bad parameters
    p = _abi.gpf_query_params(0, math.inf, 1e-6, 0)
    assert lib.gpf_radiance_fwd(h, ctypes.byref(f), ctypes.byref(q), ctypes.byref(p), fake,
                                None, None) == 5
    for bad in (_abi.gpf_query_params(3, 0.02, 1e-6, 0), _abi.gpf_query_params(0, -1.0, 1e-6, 0),
                _abi.gpf_query_params(0, 0.02, 0.0, 0), _abi.gpf_query_params(0, math.nan, 1e-6, 0)):
        assert lib.gpf_radiance_fwd(h, ctypes.byref(f), ctypes.byref(q), ctypes.byref(bad), fake,
                                    None, None) == 1
    # f64_sums: 0 or 1, and in the backward only
    p.f64_sums = 1
    assert lib.gpf_radiance_fwd(h, ctypes.byref(f), ctypes.byref(q), ctypes.byref(p), fake,
                                None, None) == 1
    assert b"f64_sums" in lib.gpf_last_error()
    p.f64_sums = 2
    g = _abi.gpf_field_grad(fake, fake, fake, fake, 0, 0)
    assert lib.gpf_radiance_bwd(h, ctypes.byref(f), ctypes.byref(q), ctypes.byref(p), fake, None,
                                None, ctypes.byref(g), None) == 1
    assert b"f64_sums" in lib.gpf_last_error()
    stats = _abi.gpf_index_stats_t()
    assert lib.gpf_index_stats(h, ctypes.byref(stats), None) == 5
    # the flags word: a device pointer on a built index
    assert lib.gpf_index_flags_async(None, fake, None) == 1
    assert lib.gpf_index_flags_async(h, None, None) == 1
    assert lib.gpf_index_flags_async(h, fake + 2, None) == 1
    assert lib.gpf_index_flags_async(h, fake, None) == 5
    # timing events: any handles (or none) on a live index, never on NULL
    assert lib.gpf_index_set_timing_events(None, None, None, None, None) == 1
    assert lib.gpf_index_set_timing_events(h, None, None, None, None) == 0
    lib.gpf_index_destroy(h)


def test_loss_and_adam_validation(lib):
    from paper_2512_12459_gb300 import _abi
    fake = 1 << 40
    sz = ctypes.c_size_t()
    assert lib.gpf_mse_workspace_size(1000, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.gpf_mse_workspace_size(-1, ctypes.byref(sz)) == 1
    assert lib.gpf_mse_loss_grad(1000, 0, fake, fake, None, fake, fake, fake, sz.value, None) == 1
    assert lib.gpf_mse_loss_grad(1000, 3, fake, fake, None, fake, fake, fake, 8, None) == 3
    f = _abi.gpf_field(10, 3, 0, fake, fake, fake, fake)
    g = _abi.gpf_field_grad(fake, fake, fake, fake, 0, 0)
    hp = _abi.gpf_adam_hparams((ctypes.c_float * 4)(5e-4, 5e-4, 5e-4, 5e-4), 0.9, 0.999, 1e-8, 0)
    assert lib.gpf_adam_step(ctypes.byref(f), ctypes.byref(g), ctypes.byref(g), ctypes.byref(g),
                             ctypes.byref(hp), None) == 1
    hp.step, hp.beta1 = 1, 1.0
    assert lib.gpf_adam_step(ctypes.byref(f), ctypes.byref(g), ctypes.byref(g), ctypes.byref(g),
                             ctypes.byref(hp), None) == 1
    # a device step counter: step must be 0 and the counter 8-byte aligned
    hp.beta1, hp.step, hp.step_counter = 0.9, 1, fake
    assert lib.gpf_adam_step(ctypes.byref(f), ctypes.byref(g), ctypes.byref(g), ctypes.byref(g),
                             ctypes.byref(hp), None) == 1
    hp.step, hp.step_counter = 0, fake + 4
    assert lib.gpf_adam_step(ctypes.byref(f), ctypes.byref(g), ctypes.byref(g), ctypes.byref(g),
                             ctypes.byref(hp), None) == 1
    assert b"step_counter" in lib.gpf_last_error()
    # a guard index must have been built
    h = ctypes.c_void_p()
    cfg = _cfg()
    assert lib.gpf_index_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    hp.step, hp.step_counter, hp.guard = 1, None, h
    assert lib.gpf_adam_step(ctypes.byref(f), ctypes.byref(g), ctypes.byref(g), ctypes.byref(g),
                             ctypes.byref(hp), None) == 5
    assert b"guard" in lib.gpf_last_error()
    lib.gpf_index_destroy(h)


def test_sort_validation(lib):
    fake = 1 << 40
    sz = ctypes.c_size_t()
    assert lib.gpf_sort_pairs_workspace_size(10_000_000, ctypes.byref(sz)) == 0
    small = sz.value
    assert lib.gpf_sort_pairs_workspace_size(20_000_000, ctypes.byref(sz)) == 0
    assert sz.value > small > 256
    assert lib.gpf_sort_pairs_workspace_size(-1, ctypes.byref(sz)) == 1
    assert lib.gpf_sort_pairs_workspace_size(1 << 31, ctypes.byref(sz)) == 1
    alt = ctypes.c_int32()
    args = (fake, fake, fake, fake, 1000)
    assert lib.gpf_sort_pairs(*args, 33, fake, 1 << 30, ctypes.byref(alt), None) == 1
    assert lib.gpf_sort_pairs(*args, 24, fake + 16, 1 << 30, ctypes.byref(alt), None) == 1
    assert lib.gpf_sort_pairs(*args, 24, fake, 16, ctypes.byref(alt), None) == 3
    assert lib.gpf_sort_pairs(None, fake, fake, fake, 1000, 24, fake, 1 << 30,
                              ctypes.byref(alt), None) == 1
    assert lib.gpf_sort_pairs(*args, 24, fake, 1 << 30, None, None) == 1
    assert lib.gpf_test_sort_wait_timeout(0, None) == 1
    assert lib.gpf_test_sort_wait_timeout((1 << 22) + 1, None) == 1


def test_package_defaults_are_the_papers(lib):
    import paper_2512_12459_gb300 as gpf
    c = load_constants()
    assert gpf.PAPER_R == c["query_radius_r"]
    assert gpf.PAPER_EPS == c["normalisation_eps"]
    assert gpf.PAPER_LR == c["adam_lr"]


def test_generators_are_seeded():
    import synth
    a = synth.config1_random(seed=3, n=50, m=60)
    b = synth.config1_random(seed=3, n=50, m=60)
    for x, y in zip((a[0].mean, a[0].quat, a[1].x), (b[0].mean, b[0].quat, b[1].x)):
        assert np.array_equal(x, y)
    pos, flux = synth.caustic_photons(2000, seed=1)
    assert pos.shape == (2000, 3) and flux.shape == (2000, 3) and np.all(flux >= 0)
    on_floor = np.abs(pos[:, 2]) < 1e-12
    assert 0.7 < on_floor.mean() < 0.99
    q = synth.pinhole_hitpoints((0, -6, 4), (0, 0, 0.5), 64, 48)
    assert q.m == 64 * 48 and q.valid.mean() > 0.4
    v = q.valid.astype(bool)
    assert np.all(np.sum(q.n[:, v] * q.wo[:, v], axis=0) > 0)
    mp, mf = synth.merge_photon_pairs(pos, flux)
    assert mp.shape[0] == 1000 and np.allclose(mf.sum(), flux.sum())


def test_box_cell_quotients_are_exact_in_float32():
    """emit_kernel recovers the cell of bit c of a box's occupied-cell mask
    (x fastest, boxes of at most 31 cells) as dz = floor((c + 0.5) / (nx ny)),
    dy = floor((r + 0.5) / nx) in float32 with correctly rounded reciprocals:
    exact for every box shape and bit index it can meet."""
    f = np.float32
    for nx in range(1, 32):
        for ny in range(1, 32):
            for nz in range(1, 32):
                if nx * ny * nz > 31:
                    continue
                nxy = nx * ny
                inx, inxy = f(1) / f(nx), f(1) / f(nxy)
                for c in range(nx * ny * nz):
                    dz = int(f(f(c) + f(0.5)) * inxy)
                    r = c - dz * nxy
                    dy = int(f(f(r) + f(0.5)) * inx)
                    assert (dz, dy, r - dy * nx) == (c // nxy, (c % nxy) // nx, c % nx)


def test_falloff_distance_newton_step_is_within_an_ulp():
    """The forward's |d| (dist_of in gpf_fwd.cu): s = d2 y with y a reciprocal
    square root of relative error up to 2^-22, then s + (y/2)(d2 - s^2) with
    the residual and the update each rounded once (fused multiply-adds).
    Emulated in float32 with exact float64 intermediates, it stays within one
    ulp of the correctly rounded square root and within u = 2^-24 relative
    of the exact one, for rsqrt errors at both ends of the range and random
    ones, which is the <= 2u the forward's exponent bound assumes."""
    rng = np.random.default_rng(7)
    d2 = (10.0 ** rng.uniform(-10, 3, 100000)).astype(np.float32)
    d64 = d2.astype(np.float64)
    root = np.sqrt(d64)
    for eps in (-2.0 ** -22, 2.0 ** -22, rng.uniform(-2.0 ** -22, 2.0 ** -22, d2.size)):
        y = (1.0 / root * (1.0 + eps)).astype(np.float32)
        s = (d64 * y).astype(np.float32)
        h = (np.float32(0.5) * y).astype(np.float32)
        res = (d64 - s.astype(np.float64) ** 2).astype(np.float32)
        s1 = (h.astype(np.float64) * res.astype(np.float64) + s.astype(np.float64)).astype(np.float32)
        rn = root.astype(np.float32)
        assert np.all(np.abs(s1.astype(np.float64) - rn) <= np.spacing(rn))
        assert np.max(np.abs(s1.astype(np.float64) - root) / root) <= 2.0 ** -24 * 1.001
