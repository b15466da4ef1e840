"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function that include/mvd.h declares, rejects bad arguments before any
device work, and factorises PSFs the way the kernels expect."""

import ctypes

import numpy as np
import pytest

from paper_1503_07998_gb300 import build as B
from paper_1503_07998_gb300 import mvd, synth


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    return mvd.lib()


def test_exports_every_header_function():
    names = mvd.header_functions()
    assert "mvd_create" in names and "mvd_deconvolve_planes" in names and "mvd_reslice" in names
    missing = [n for n in names if not hasattr(mvd.lib(), n)]
    assert not missing, missing


def test_status_strings():
    assert mvd.mvd_status_string(0) == "ok"
    assert "argument" in mvd.mvd_status_string(1)
    assert mvd.mvd_status_string(99) == "unknown status"


def _create(views=2, K=5, H=16, W=16, iters=3, boundary=0, eps=1e-6, psfs=None):
    if psfs is None:
        psfs = np.full((max(views, 1), max(K, 1), max(K, 1)), 0.1, dtype=np.float32)
    h = ctypes.c_void_p()
    st = mvd.lib().mvd_create(ctypes.byref(h), views, psfs.ctypes.data_as(ctypes.c_void_p), K, H, W, iters,
                              boundary, eps)
    return st, h


@pytest.mark.parametrize("kw", [
    dict(K=4), dict(K=0), dict(views=0), dict(views=65), dict(H=0), dict(iters=-1),
    dict(eps=0.0), dict(eps=-1.0), dict(eps=float("inf")), dict(K=17, boundary=1), dict(boundary=7),
])
def test_create_rejects_bad_arguments(kw):
    st, h = _create(**kw)
    assert st == mvd.MVD_ERR_ARG, (kw, st, mvd.mvd_last_error())
    assert h.value is None
    assert mvd.mvd_last_error() != ""


@pytest.mark.parametrize("bad", ["negative", "nan", "zero"])
def test_create_rejects_bad_psfs(bad):
    p = np.full((2, 3, 3), 0.1, dtype=np.float32)
    if bad == "negative":
        p[1, 0, 0] = -0.01
    elif bad == "nan":
        p[0, 1, 1] = np.nan
    else:
        p[1] = 0
    st, _ = _create(K=3, psfs=p)
    assert st == mvd.MVD_ERR_ARG


def _reconstruct(taps, ranks, K, views, shared):
    """Sum of outer products per view from the correlation-order factors."""
    out, off = [], 0
    seen = {}
    for v in range(views):
        if shared[v] in seen:
            out.append(out[seen[shared[v]]])
            continue
        seen[shared[v]] = v
        P = np.zeros((K, K))
        for q in range(ranks[v]):
            u = taps[off + q, 2].astype(np.float64)
            w = taps[off + q, 3].astype(np.float64)
            np.testing.assert_array_equal(taps[off + q, 0], taps[off + q, 2][::-1])
            np.testing.assert_array_equal(taps[off + q, 1], taps[off + q, 3][::-1])
            P += np.outer(u, w)
        off += ranks[v]
        out.append(P)
    return out


def test_gaussian_psfs_are_rank_one():
    psfs = np.stack([synth.gaussian_psf(31, 8.0, 1.5, a) for a in (0, 90, 180, 270)])
    ranks, taps = mvd.mvd_psf_factors(psfs)
    assert list(ranks) == [1, 1, 1, 1]
    rec = _reconstruct(taps, ranks, 31, 4, [0, 1, 0, 1])
    for v in range(4):
        P = psfs[v].astype(np.float64)
        assert np.linalg.norm(rec[v] - P) <= 1e-6 * np.linalg.norm(P)


def test_general_psf_full_rank_reconstructs():
    rng = np.random.default_rng(0)
    psfs = rng.random((2, 9, 9)).astype(np.float32)
    ranks, taps = mvd.mvd_psf_factors(psfs, rank_tol=0.0)
    assert list(ranks) == [9, 9]
    rec = _reconstruct(taps, ranks, 9, 2, [0, 1])
    for v in range(2):
        P = psfs[v].astype(np.float64)
        assert np.linalg.norm(rec[v] - P) <= 1e-6 * np.linalg.norm(P)
    # the default tolerance keeps every term a random PSF needs
    r2, t2 = mvd.mvd_psf_factors(psfs)
    rec2 = _reconstruct(t2, r2, 9, 2, [0, 1])
    for v in range(2):
        assert np.linalg.norm(rec2[v] - psfs[v]) <= 1e-6 * np.linalg.norm(psfs[v])


def test_rotated_gaussian_needs_several_terms():
    psfs = synth.gaussian_psf(17, 5.0, 1.2, 30.0)[None]
    ranks, taps = mvd.mvd_psf_factors(psfs)
    assert 1 < ranks[0] <= 17
    rec = _reconstruct(taps, ranks, 17, 1, [0])
    assert np.linalg.norm(rec[0] - psfs[0]) <= 1e-6 * np.linalg.norm(psfs[0])


@pytest.mark.parametrize("variant", ["independent", "efficient_bayesian", "optimization_1", "optimization_2"])
def test_variant_kernels_match_oracle(variant):
    """The library's host-built X_v (FP64, rounded to FP32) equal the oracle's
    on non-symmetric PSFs of three views and on oblique Gaussians."""
    import oracle
    rng = np.random.default_rng(21)
    for psfs in (rng.random((3, 7, 7)).astype(np.float32) + 0.05,
                 np.stack([synth.gaussian_psf(15, 3.0, 1.0, a) for a in (0, 60, 120)])):
        got = mvd.mvd_variant_kernels(psfs, variant)
        want = oracle.correlation_kernels(psfs.astype(np.float64), variant)
        np.testing.assert_allclose(got, want, rtol=2e-6, atol=1e-7 * want.max())


def test_variant_rejects_bad_arguments():
    psfs = np.ones((2, 5, 5), np.float32)
    with pytest.raises(KeyError):
        mvd.mvd_variant_kernels(psfs, "nope")
    bad = psfs.copy()
    bad[0, 0, 0] = -1
    with pytest.raises(mvd.MvdError):
        mvd.mvd_variant_kernels(bad, "optimization_2")
    out = np.zeros_like(psfs)
    st = mvd.lib().mvd_variant_kernels(psfs.ctypes.data_as(ctypes.c_void_p), 2, 5, 7,
                                       out.ctypes.data_as(ctypes.c_void_p))
    assert st == mvd.MVD_ERR_ARG


def test_host_chunks_uniform_and_small_volumes():
    assert mvd.mvd_host_chunks(37, 7680, 8) == [(0, 8), (8, 8), (16, 8), (24, 8), (32, 5)]
    # small volume, automatic: four equal chunks
    assert mvd.mvd_host_chunks(37, 7680, 0) == [(0, 10), (10, 10), (20, 10), (30, 7)]
    assert mvd.mvd_host_chunks(1, 1 << 20, 0) == [(0, 1)]
    assert mvd.mvd_host_chunks(3, 1 << 20, 5) == [(0, 3)]


def test_host_chunks_ramp_for_large_volumes():
    # 1024 planes of 8 MiB (4 views of 1024 x 1024 uint16): base 128 planes
    # (1 GiB); ramp 16, 32, 64; 880 planes in 7 middle chunks; last 32
    ch = mvd.mvd_host_chunks(1024, 8 << 20, 0)
    sizes = [n for _, n in ch]
    assert sizes[:3] == [16, 32, 64] and sizes[-1] == 32
    assert len(sizes) == 11 and all(125 <= n <= 128 for n in sizes[3:-1]) and sum(sizes) == 1024
    # 2048 planes of 1 MiB: base 512 (a quarter of the volume); ramp 64, 128,
    # 256; 1472 planes in 3 middle chunks; last 128
    assert [n for _, n in mvd.mvd_host_chunks(2048, 1 << 20, 0)] == [64, 128, 256, 491, 491, 490, 128]
    # 512 planes of 1 MiB (2 views of 512 x 512 uint16): base 128
    assert [n for _, n in mvd.mvd_host_chunks(512, 1 << 20, 0)] == [16, 32, 64, 123, 123, 122, 32]
    # 4096 planes of 1 MiB: ramp 128, 256, 512; 2944 planes in 3 middle chunks; last 256
    assert [n for _, n in mvd.mvd_host_chunks(4096, 1 << 20, 0)] == [128, 256, 512, 982, 981, 981, 256]
    # planes above 128 MiB (base under 8 planes): four equal chunks
    assert mvd.mvd_host_chunks(40, 256 << 20, 0) == [(0, 10), (10, 10), (20, 10), (30, 10)]
    # under 256 MiB of input: four equal chunks
    assert mvd.mvd_host_chunks(200, 1 << 20, 0) == [(0, 50), (50, 50), (100, 50), (150, 50)]


def test_host_chunks_cover_every_plane_once():
    rng = np.random.default_rng(3)
    for _ in range(300):
        ny = int(rng.integers(1, 3000))
        pb = int(rng.integers(1, 1 << 24))
        cp = int(rng.integers(0, 50)) if rng.random() < 0.5 else 0
        ch = mvd.mvd_host_chunks(ny, pb, cp)
        y = 0
        for y0, n in ch:
            assert y0 == y and n >= 1
            if cp:
                assert n <= cp
            y += n
        assert y == ny


def test_host_chunks_rejects_bad_arguments():
    for args in ((0, 100, 0), (5, 0, 0), (5, 100, -1)):
        with pytest.raises(mvd.MvdError):
            mvd.mvd_host_chunks(*args)
    y0 = np.zeros(2, dtype=np.int32)
    n = np.zeros(2, dtype=np.int32)
    # three chunks do not fit two slots
    assert mvd.lib().mvd_host_chunks(30, 100, 10, y0.ctypes.data_as(ctypes.c_void_p),
                                     n.ctypes.data_as(ctypes.c_void_p), 2) == -1


@pytest.mark.parametrize("bad", ["zero_sum", "negative", "nan"])
def test_static_entry_point_rejects_bad_psfs_before_device_work(bad):
    """mvd_deconvolve_planes_static checks its PSFs as mvd_create does, before
    it touches the device: the buffer addresses passed here are never used."""
    p = np.full((2, 5, 5), 0.04, dtype=np.float32)
    if bad == "zero_sum":
        p[1] = 0.0
    elif bad == "negative":
        p[0, 2, 2] = -1e-3
    else:
        p[1, 0, 4] = np.nan
    fake_data, fake_est = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 30)
    st = mvd.lib().mvd_deconvolve_planes_static(2, p.ctypes.data_as(ctypes.c_void_p), 5, 16, 16, 3, 0, 1e-6,
                                                fake_data, mvd.DTYPE["f32"], fake_est, 1, 1, None)
    assert st == mvd.MVD_ERR_ARG, (bad, st)
    assert "PSF" in mvd.mvd_last_error()


def test_allocation_failure_hook_arguments():
    assert mvd.lib().mvd_debug_fail_allocations(-1) == mvd.MVD_ERR_ARG
    assert mvd.lib().mvd_debug_fail_allocations(0) == mvd.MVD_OK
    assert mvd.lib().mvd_static_set_wait_budget(0) == mvd.MVD_OK
