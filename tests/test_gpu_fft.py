"""Parity of the Fourier route (MVD_ALGO_FFT: the library's own mixed-radix
FFT with fused pointwise steps) with the FP64 oracle."""

import json
import os

import numpy as np
import pytest

import oracle
from paper_1503_07998_gb300 import synth
from tests.parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def mvd():
    from paper_1503_07998_gb300 import build as B
    B.build()
    from paper_1503_07998_gb300 import mvd as m
    m.lib()
    return m


def run_fft(mvd, phi, psfs, iters, boundary="zero", order="simultaneous", psi0=None):
    V, P, H, W = phi.shape
    ctx = mvd.mvd_create(V, psfs, psfs.shape[-1], H, W, iters, boundary, 1e-6)
    try:
        mvd.mvd_set_algo(ctx, "fft")
        mvd.mvd_set_update_order(ctx, order)
        d = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
        if psi0 is None:
            est = torch.empty((P, H, W), device="cuda")
        else:
            est = torch.from_numpy(np.ascontiguousarray(psi0, dtype=np.float32)).cuda()
        mvd.mvd_deconvolve_planes(ctx, d, est, init_mean=psi0 is None)
        torch.cuda.synchronize()
        return est.cpu().numpy()
    finally:
        ctx.close()


def test_golden_small_zero(mvd):
    with open(os.path.join(GOLDEN, "small_zero.json")) as f:
        case = json.load(f)
    got = run_fft(mvd, np.array(case["phi"], np.float32), np.array(case["psf"], np.float32), case["iters"])
    assert_parity(got, np.array(case["expected"]), what="fft golden")


def test_single_plane_two_views_k17(mvd):
    c = synth.plane_case(seed=0)
    ref = oracle.rl_planes(c.phi, c.psfs, c.iters, eps=c.eps, route="fft")
    assert_parity(run_fft(mvd, c.phi, c.psfs, c.iters), ref, what="fft plane")


@pytest.mark.parametrize("dtype", [np.uint16, np.float32])
def test_oblique_views_sequential(mvd, dtype):
    """Four views at 0/45/90/135 degrees: the turned PSFs have SVD rank ~30."""
    c = synth.plane_case(seed=8, H=150, W=200, n_planes=2, n_blobs=60, K=31, sigma_axial=8.0,
                         sigma_lateral=1.5, angles=(0, 45, 90, 135), dtype=dtype)
    ref = oracle.rl_planes(c.phi, c.psfs, 5, eps=1e-6, route="fft", order="sequential")
    assert_parity(run_fft(mvd, c.phi, c.psfs, 5, order="sequential"), ref, what="fft oblique")


def test_psf_larger_than_the_fused_kernels_take(mvd):
    c = synth.plane_case(seed=9, H=100, W=120, n_planes=3, n_blobs=40, K=63, sigma_axial=14.0,
                         sigma_lateral=2.0, dtype=np.uint16)
    ref = oracle.rl_planes(c.phi, c.psfs, 4, eps=1e-6, route="fft")
    assert_parity(run_fft(mvd, c.phi, c.psfs, 4), ref, what="fft K=63")


def test_circular_boundary_on_smooth_sizes(mvd):
    rng = np.random.default_rng(90)
    psfs = (rng.random((2, 15, 15)) + 0.05).astype(np.float32)
    psfs /= psfs.sum(axis=(1, 2), keepdims=True)
    phi = rng.uniform(20, 300, size=(2, 2, 96, 120)).astype(np.float32)
    ref = oracle.rl_planes(phi, psfs, 3, boundary="circular", route="fft")
    assert_parity(run_fft(mvd, phi, psfs, 3, boundary="circular"), ref, what="fft circular")


def test_given_start_and_agreement_with_fused(mvd):
    c = synth.plane_case(seed=10, H=64, W=96, n_planes=2, n_blobs=30, K=17, sigma_axial=5.0,
                         sigma_lateral=1.3, dtype=np.float32)
    psi0 = np.full((2, 64, 96), 30.0, np.float32)
    ref = oracle.rl_planes(c.phi, c.psfs, 3, psi0=psi0.astype(np.float64))
    assert_parity(run_fft(mvd, c.phi, c.psfs, 3, psi0=psi0), ref, what="fft psi0")


def test_autotune_picks_a_route_and_keeps_parity(mvd, tmp_path, monkeypatch):
    monkeypatch.setenv("MVD_TUNE_CACHE", str(tmp_path / "tune.txt"))
    c = synth.plane_case(seed=11, H=160, W=160, n_planes=4, n_blobs=50, K=31, sigma_axial=8.0,
                         sigma_lateral=1.5, angles=(0, 45), dtype=np.uint16)
    V, P, H, W = c.phi.shape
    ctx = mvd.mvd_create(V, c.psfs, 31, H, W, 4, "zero", 1e-6)
    try:
        d = torch.from_numpy(c.phi).cuda()
        route = mvd.mvd_autotune(ctx, d)
        assert route in ("fused", "fft")
        assert "route_" in (tmp_path / "tune.txt").read_text()
        assert mvd.mvd_autotune(ctx, d) == route          # from the cache
        est = torch.empty((P, H, W), device="cuda")
        mvd.mvd_deconvolve_planes(ctx, d, est)
        torch.cuda.synchronize()
    finally:
        ctx.close()
    ref = oracle.rl_planes(c.phi, c.psfs, 4, eps=1e-6, route="fft")
    assert_parity(est.cpu().numpy(), ref, what=f"autotuned ({route})")


def test_injected_copy_timeout_is_reported_and_context_recovers(mvd):
    """The ratio pass prefetches each job's rows with bulk async copies on
    bounded mbarrier waits: a negative wait budget makes them report a
    timeout (MVD_ERR_TIMEOUT) once the copies land; with the default budget
    the same context is correct."""
    c = synth.plane_case(seed=12, H=96, W=128, n_planes=2, n_blobs=40, K=21, sigma_axial=5.0,
                         sigma_lateral=1.4, dtype=np.uint16)
    V, P, H, W = c.phi.shape
    ctx = mvd.mvd_create(V, c.psfs, 21, H, W, 3, "zero", 1e-6)
    try:
        mvd.mvd_set_algo(ctx, "fft")
        d = torch.from_numpy(c.phi).cuda()
        est = torch.empty((P, H, W), device="cuda")
        mvd.mvd_set_wait_budget(ctx, -1)
        mvd.mvd_deconvolve_planes(ctx, d, est)
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_device_status(ctx)
        assert ei.value.status == mvd.MVD_ERR_TIMEOUT
        mvd.mvd_set_wait_budget(ctx, 0)
        mvd.mvd_deconvolve_planes(ctx, d, est)
        mvd.mvd_device_status(ctx)
        got = est.cpu().numpy()
    finally:
        ctx.close()
    ref = oracle.rl_planes(c.phi, c.psfs, 3, eps=1e-6, route="fft")
    assert_parity(got, ref, what="fft after an injected timeout")
