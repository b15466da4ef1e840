"""Parity of the tensor-core route's warp-specialised kernels (tcw_*) with
the FP64 oracle.  The tensor route (MVD_ALGO_TENSOR, BF16x3 tcgen05 passes,
FP32 ratio and update) runs a launch on them when its views share one rank-1
factorisation on the zero boundary: every launch of the sequential update
order with Gaussian PSFs, and the blur of views with identical PSFs in the
simultaneous order.  Each case checks, through the profiler's kernel names,
that those kernels did run, and compares with the oracle at the FP32
tolerances (rel-L2 1e-4, per pixel 1e-3)."""

import numpy as np
import pytest

import oracle
from paper_1503_07998_gb300 import synth
from tests.parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mvd():
    from paper_1503_07998_gb300 import build as B
    B.build()
    from paper_1503_07998_gb300 import mvd as m
    m.lib()
    return m


def run_ws(mvd, phi, psfs, iters, order="sequential", psi0=None, expect=("tcw_blur_ratio", "tcw_correlate_update")):
    V, P, H, W = phi.shape
    K = psfs.shape[-1]
    ctx = mvd.mvd_create(V, psfs, K, H, W, iters, "zero", 1e-6)
    try:
        mvd.mvd_set_algo(ctx, "tensor")
        mvd.mvd_set_update_order(ctx, order)
        d = torch.from_numpy(np.ascontiguousarray(phi)).to(DEV)
        if psi0 is None:
            est = torch.empty((P, H, W), dtype=torch.float32, device=DEV)
        else:
            est = torch.from_numpy(np.ascontiguousarray(psi0, dtype=np.float32)).to(DEV)
        mvd.mvd_profile_enable(ctx, True)
        mvd.mvd_deconvolve_planes(ctx, d, est, init_mean=psi0 is None)
        torch.cuda.synchronize()
        mvd.mvd_device_status(ctx)
        prof = mvd.mvd_profile_read(ctx)
        for name in expect:
            assert name in prof, (name, sorted(prof))
        return est.cpu().numpy()
    finally:
        ctx.close()


@pytest.mark.parametrize("K", [1, 3, 9, 17, 31, 41, 47])
def test_sequential_views_every_psf_size(mvd, K):
    """Two views at 0/90 degrees, ragged 200 x 172 planes (partial tiles in
    both directions), uint16 data, 4 iterations in sequence."""
    sa = max(1.0, K / 5.0)
    c = synth.plane_case(seed=100 + K, H=200, W=172, n_planes=2, n_blobs=60, K=K, sigma_axial=sa,
                         sigma_lateral=min(1.5, sa), iters=4, dtype=np.uint16)
    ref = oracle.rl_planes(c.phi, c.psfs, 4, eps=1e-6, route="fft", order="sequential")
    assert_parity(run_ws(mvd, c.phi, c.psfs, 4), ref, what=f"tcw K={K}")


@pytest.mark.parametrize("dtype", [np.uint16, np.float32])
def test_four_views_k41_several_tiles(mvd, dtype):
    """Four views at 0/90/180/270 degrees, 41x41 PSFs sigma (1.8, 10), three
    planes of 300 x 260 (three by three tiles, ragged), 10 iterations in
    sequence: the precision workload's PSFs on a small volume."""
    c = synth.plane_case(seed=110, H=300, W=260, n_planes=3, n_blobs=120, K=41, sigma_axial=10.0,
                         sigma_lateral=1.8, angles=(0, 90, 180, 270), iters=10, dtype=dtype)
    ref = oracle.rl_planes(c.phi, c.psfs, 10, eps=1e-6, route="fft", order="sequential")
    assert_parity(run_ws(mvd, c.phi, c.psfs, 10), ref, what="tcw 4 views K=41")


def test_whole_tiles_and_a_tiny_plane(mvd):
    """Planes of exactly 256 x 256 (whole tiles only) and of 40 x 36 (one
    tile, mostly outside the plane)."""
    for H, W, n in ((256, 256, 2), (40, 36, 3)):
        c = synth.plane_case(seed=120 + H, H=H, W=W, n_planes=n, n_blobs=max(10, H * W // 800), K=15,
                             sigma_axial=3.0, sigma_lateral=1.3, iters=5, dtype=np.float32)
        ref = oracle.rl_planes(c.phi, c.psfs, 5, eps=1e-6, route="fft", order="sequential")
        assert_parity(run_ws(mvd, c.phi, c.psfs, 5), ref, what=f"tcw {H}x{W}")


def test_given_initial_estimate(mvd):
    """init_mean off: the first iteration's blur reads the given estimate
    through TMA (the constant-estimate path is the default elsewhere)."""
    c = synth.plane_case(seed=130, H=150, W=136, n_planes=2, n_blobs=50, K=21, sigma_axial=5.0,
                         sigma_lateral=1.4, iters=3, dtype=np.float32)
    psi0 = np.random.default_rng(130).uniform(20, 60, size=(2, 150, 136))
    ref = oracle.rl_planes(c.phi, c.psfs, 3, eps=1e-6, psi0=psi0, route="fft", order="sequential")
    assert_parity(run_ws(mvd, c.phi, c.psfs, 3, psi0=psi0), ref, what="tcw given estimate")


def test_simultaneous_views_with_one_psf(mvd):
    """Two views that share one PSF in the simultaneous order: their blur is
    one warp-specialised launch writing both ratios; the correlation of two
    views runs on the lock-step tensor kernel."""
    c = synth.plane_case(seed=140, H=180, W=200, n_planes=2, n_blobs=60, K=25, sigma_axial=6.0,
                         sigma_lateral=1.5, angles=(0, 180), iters=4, dtype=np.uint16)
    ref = oracle.rl_planes(c.phi, c.psfs, 4, eps=1e-6, route="fft")
    got = run_ws(mvd, c.phi, c.psfs, 4, order="simultaneous", expect=("tcw_blur_ratio", "tc_correlate_update"))
    assert_parity(got, ref, what="tcw simultaneous, one PSF")


def test_injected_wait_timeout_is_reported_and_context_recovers(mvd):
    """A negative wait budget makes every bounded wait of the warp-specialised
    kernels report a timeout once its event has come: the CTA stops, drains
    its copies and MMAs, frees its tensor memory, and the host sees
    MVD_ERR_TIMEOUT; with the default budget the same context is correct."""
    c = synth.plane_case(seed=150, H=160, W=144, n_planes=2, n_blobs=40, K=13, sigma_axial=3.0,
                         sigma_lateral=1.2, iters=3, dtype=np.float32)
    V, P, H, W = c.phi.shape
    ctx = mvd.mvd_create(V, c.psfs, 13, H, W, 3, "zero", 1e-6)
    try:
        mvd.mvd_set_algo(ctx, "tensor")
        mvd.mvd_set_update_order(ctx, "sequential")
        d = torch.from_numpy(c.phi).to(DEV)
        est = torch.empty((P, H, W), device=DEV)
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
    ref = oracle.rl_planes(c.phi, c.psfs, 3, eps=1e-6, route="fft", order="sequential")
    assert_parity(got, ref, what="tcw after an injected timeout")
