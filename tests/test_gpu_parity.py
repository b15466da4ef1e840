"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every case feeds the same seeded inputs to both sides and compares every
output pixel at the tolerances in ``tests/parity.py``.  Sizes span several
output tiles with ragged edges; the full-size volume case checks sampled
planes of the exact workload and launch configuration that bench.py times.
"""

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
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mvd():
    from paper_1503_07998_gb300 import build as B
    B.build()
    from paper_1503_07998_gb300 import mvd as m
    m.lib()
    return m


def run_gpu(mvd, phi, psfs, iters, boundary="zero", eps=1e-6, algo="fused", psi0=None, rank_tol=None,
            order="simultaneous"):
    V, P, H, W = phi.shape
    K = psfs.shape[-1]
    ctx = mvd.mvd_create(V, psfs, K, H, W, iters, boundary, eps)
    try:
        try:
            mvd.mvd_set_algo(ctx, algo)
        except mvd.MvdError as e:
            # PSFs needing more separable terms than the fused kernels carry
            # run on the plain path
            if algo != "fused" or e.status != mvd.MVD_ERR_UNSUPPORTED:
                raise
            mvd.mvd_set_algo(ctx, "plain")
        mvd.mvd_set_update_order(ctx, order)
        if rank_tol is not None:
            mvd.mvd_set_rank_tolerance(ctx, rank_tol)
        d = torch.from_numpy(np.ascontiguousarray(phi)).to(DEV)
        if psi0 is None:
            est = torch.empty((P, H, W), dtype=torch.float32, device=DEV)
        else:
            est = torch.from_numpy(np.ascontiguousarray(psi0, dtype=np.float32)).to(DEV)
        mvd.mvd_deconvolve_planes(ctx, d, est, init_mean=psi0 is None)
        torch.cuda.synchronize()
        mvd.mvd_device_status(ctx)
        return est.cpu().numpy()
    finally:
        ctx.close()


@pytest.mark.parametrize("name", ["small_zero", "small_circular"])
@pytest.mark.parametrize("algo", ["fused", "plain", "direct"])
def test_golden_fixtures(mvd, name, algo):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        case = json.load(f)
    phi = np.array(case["phi"], dtype=np.float32)
    psf = np.array(case["psf"], dtype=np.float32)
    got = run_gpu(mvd, phi, psf, case["iters"], case["boundary"], case["eps"], algo)
    assert_parity(got, np.array(case["expected"]), what=f"{name}/{algo}")


def test_hand_derived_case(mvd):
    with open(os.path.join(GOLDEN, "hand_1x3.json")) as f:
        case = json.load(f)
    phi = np.array(case["phi"], dtype=np.float32)[:, None]
    psf = np.array(case["psf"], dtype=np.float32)
    expected = np.array([[n / d for n, d in row] for row in case["expected"]])[None]
    for algo in ("fused", "plain", "direct"):
        got = run_gpu(mvd, phi, psf, 1, "zero", 1e-6, algo)
        np.testing.assert_allclose(got, expected, rtol=2e-6)


def test_single_plane_two_views_k17(mvd):
    """One 128x128 FP32 plane, 2 views, 17x17 sigma (1.5, 6) PSFs turned by
    90 degrees, 200 blobs, seed 0, zero boundary, eps 1e-6, 10 iterations."""
    c = synth.plane_case(seed=0)
    ref = oracle.rl_planes(c.phi, c.psfs, c.iters, boundary="zero", eps=c.eps, route="fft")
    for algo in ("fused", "plain"):
        got = run_gpu(mvd, c.phi, c.psfs, c.iters, "zero", c.eps, algo)
        assert_parity(got, ref, what=f"plane/{algo}")


@pytest.mark.parametrize("boundary", ["zero", "circular"])
@pytest.mark.parametrize("K,V,H,W,dtype", [
    (1, 1, 33, 47, np.float32),
    (3, 3, 70, 150, np.uint16),
    (17, 2, 130, 260, np.uint16),
    (31, 2, 97, 141, np.float32),
    (41, 4, 150, 135, np.uint16),
    (47, 1, 64, 256, np.float32),
])
def test_ragged_tiles_general_psfs(mvd, boundary, K, V, H, W, dtype):
    """Random non-symmetric PSFs (full SVD rank), several tiles, ragged edges."""
    if boundary == "circular" and K > min(H, W):
        pytest.skip("circular needs K <= plane")
    rng = np.random.default_rng(K * 1000 + V)
    psfs = (rng.random((V, K, K)) + 0.05).astype(np.float32)
    psfs /= psfs.sum(axis=(1, 2), keepdims=True)
    P = 2
    base = rng.uniform(20, 400, size=(V, P, H, W))
    phi = base.astype(dtype) if dtype == np.float32 else np.round(base).astype(np.uint16)
    iters = 3
    ref = oracle.rl_planes(phi, psfs, iters, boundary=boundary, eps=1e-6, route="fft")
    got = run_gpu(mvd, phi, psfs, iters, boundary)
    assert_parity(got, ref, what=f"fused K={K} V={V} {boundary}")


@pytest.mark.parametrize("boundary", ["zero", "circular"])
@pytest.mark.parametrize("K,angles,H,W", [(41, (0, 90, 180, 270), 150, 135), (47, (0, 90), 64, 256),
                                          (45, (0, 90, 45), 100, 200)])
def test_fused_large_psfs_few_terms(mvd, boundary, K, angles, H, W):
    """Gaussian PSFs (one term when axis-aligned, a few when turned by 45
    degrees) at the largest sizes the fused kernels take."""
    c = synth.plane_case(seed=K, H=H, W=W, n_planes=2, n_blobs=50, K=K, sigma_axial=9.0,
                         sigma_lateral=1.8, angles=angles, dtype=np.uint16)
    ctx = mvd.mvd_create(len(angles), c.psfs, K, H, W, 3, boundary, 1e-6)
    try:
        mvd.mvd_set_algo(ctx, "fused")          # must be available
    finally:
        ctx.close()
    order = "sequential" if len(angles) > 2 else "simultaneous"
    ref = oracle.rl_planes(c.phi, c.psfs, 3, boundary=boundary, eps=1e-6, route="fft", order=order)
    got = run_gpu(mvd, c.phi, c.psfs, 3, boundary, order=order)
    assert_parity(got, ref, what=f"fused K={K} views={len(angles)} {boundary}")


@pytest.mark.parametrize("boundary", ["zero", "circular"])
@pytest.mark.parametrize("algo", ["fused", "plain"])
def test_four_views_sequential_order(mvd, boundary, algo):
    """Views at 0/90/180/270 degrees (two distinct in-plane PSFs, rank one),
    each view updating the estimate in turn."""
    c = synth.plane_case(seed=3, H=200, W=168, n_planes=3, n_blobs=40, K=41, sigma_axial=10.0,
                         sigma_lateral=1.8, angles=(0, 90, 180, 270), dtype=np.uint16)
    info_ctx = mvd.mvd_create(4, c.psfs, 41, 200, 168, 10, boundary, 1e-6)
    info = mvd.mvd_get_info(info_ctx)
    info_ctx.close()
    assert info.rank == [1, 1, 1, 1] and info.blur_groups == 2 and info.blur_terms == 2
    ref = oracle.rl_planes(c.phi, c.psfs, 10, boundary=boundary, eps=1e-6, route="fft", order="sequential")
    got = run_gpu(mvd, c.phi, c.psfs, 10, boundary, algo=algo, order="sequential")
    assert_parity(got, ref, what=f"4 views sequential {boundary} {algo}")


def test_shared_psf_blurred_once_simultaneous(mvd):
    """Views 180 degrees apart share one PSF: kernel A blurs once for both."""
    c = synth.plane_case(seed=4, H=130, W=150, n_planes=2, n_blobs=60, K=31, sigma_axial=8.0,
                         sigma_lateral=1.5, angles=(0, 180), dtype=np.uint16)
    ref = oracle.rl_planes(c.phi, c.psfs, 3, eps=1e-6, route="fft")
    got = run_gpu(mvd, c.phi, c.psfs, 3)
    assert_parity(got, ref, what="shared PSF")


def test_given_initial_estimate_and_zero_iterations(mvd):
    rng = np.random.default_rng(5)
    V, P, H, W, K = 2, 2, 40, 70, 7
    psfs = (rng.random((V, K, K)) + 0.1).astype(np.float32)
    phi = rng.uniform(5, 50, size=(V, P, H, W)).astype(np.float32)
    psi0 = rng.uniform(5, 50, size=(P, H, W)).astype(np.float32)
    for iters in (1, 2, 3):
        ref = oracle.rl_planes(phi, psfs, iters, psi0=psi0.astype(np.float64))
        for algo in ("fused", "plain"):
            got = run_gpu(mvd, phi, psfs, iters, algo=algo, psi0=psi0)
            assert_parity(got, ref, what=f"psi0 iters={iters} {algo}")
    got = run_gpu(mvd, phi, psfs, 0)
    np.testing.assert_allclose(got, np.broadcast_to(oracle.init_mean(phi)[:, None, None], got.shape), rtol=1e-6)


def test_mean_of_uint16_planes_is_exact(mvd):
    rng = np.random.default_rng(6)
    phi = rng.integers(0, 65536, size=(3, 4, 64, 72), dtype=np.uint16)
    psfs = np.ones((3, 1, 1), dtype=np.float32)
    got = run_gpu(mvd, phi, psfs, 0)
    exact = phi.astype(np.float64).mean(axis=(0, 2, 3)).astype(np.float32)
    np.testing.assert_array_equal(got[:, 0, 0], exact)


@pytest.mark.parametrize("dtype", [torch.uint16, torch.float32])
def test_reslice_bit_exact(mvd, dtype):
    ctx = mvd.mvd_create(1, np.ones((1, 1, 1), np.float32), 1, 8, 8, 1)
    try:
        for shape in [(2, 13, 7, 24), (1, 5, 9, 11), (3, 16, 32, 64)]:
            src = torch.randint(0, 60000, shape, device=DEV, dtype=torch.int32).to(dtype)
            V, Z, Y, X = shape
            dst = torch.empty((V, Y, Z, X), dtype=dtype, device=DEV)
            mvd.mvd_reslice(ctx, src, dst)
            torch.cuda.synchronize()
            expect = oracle.reslice(src[0].cpu().to(torch.float32).numpy())
            assert np.array_equal(dst[0].cpu().to(torch.float32).numpy(), expect)
            assert torch.equal(dst.to(torch.float32), src.to(torch.float32).permute(0, 2, 1, 3))
    finally:
        ctx.close()


def test_host_pipeline_equals_device_path(mvd):
    stacks, psfs = synth.volume_stacks(40, 37, 48, 9, 4.0, 1.5, (0, 90), 5e-3, seed=11, device=DEV)
    V, Z, Y, X = stacks.shape
    ctx = mvd.mvd_create(V, psfs, 9, Z, X, 5, "zero", 1e-6)
    try:
        planes = torch.empty((V, Y, Z, X), dtype=stacks.dtype, device=DEV)
        mvd.mvd_reslice(ctx, stacks, planes)
        est = torch.empty((Y, Z, X), dtype=torch.float32, device=DEV)
        mvd.mvd_deconvolve_planes(ctx, planes, est)
        torch.cuda.synchronize()
        host_in = stacks.cpu().pin_memory()
        host_out = torch.empty((Y, Z, X), dtype=torch.float32).pin_memory()
        mvd.mvd_run_host(ctx, host_in, host_out, chunk_planes=8)
        assert torch.equal(host_out, est.cpu())
    finally:
        ctx.close()
    ref = oracle.rl_planes(planes.cpu().to(torch.int32).numpy(), psfs, 5, planes=[0, 17, 36])
    assert_parity(est.cpu().numpy()[[0, 17, 36]], ref, what="volume planes")


def test_host_pipeline_automatic_chunks_equal_device_path(mvd):
    """300 MiB of input (2 views, 1200 planes of 128 x 512): the automatic
    schedule ramps (chunks of 37, 75 and 150 planes, three of about 288, a
    last one of 75); the result equals the device path bit for bit."""
    stacks, psfs = synth.volume_stacks(128, 1200, 512, 9, 4.0, 1.5, (0, 90), 1e-4, seed=12, device=DEV)
    V, Z, Y, X = stacks.shape
    chunks = mvd.mvd_host_chunks(Y, V * Z * X * 2)
    sizes = [n for _, n in chunks]
    assert sizes[:3] == [37, 75, 150] and sizes[-1] == 75 and max(sizes) == 288 and sum(sizes) == Y
    ctx = mvd.mvd_create(V, psfs, 9, Z, X, 3, "zero", 1e-6)
    try:
        planes = torch.empty((V, Y, Z, X), dtype=stacks.dtype, device=DEV)
        mvd.mvd_reslice(ctx, stacks, planes)
        est = torch.empty((Y, Z, X), dtype=torch.float32, device=DEV)
        mvd.mvd_deconvolve_planes(ctx, planes, est)
        torch.cuda.synchronize()
        host_in = stacks.cpu().pin_memory()
        host_out = torch.empty((Y, Z, X), dtype=torch.float32).pin_memory()
        mvd.mvd_run_host(ctx, host_in, host_out)
        assert torch.equal(host_out, est.cpu())
    finally:
        ctx.close()


def test_launch_count_and_errors(mvd):
    rng = np.random.default_rng(7)
    psfs = (rng.random((2, 5, 5)) + 0.1).astype(np.float32)
    ctx = mvd.mvd_create(2, psfs, 5, 20, 30, 4)
    try:
        d = torch.ones((2, 3, 20, 30), device=DEV)
        e = torch.empty((3, 20, 30), device=DEV)
        n0 = mvd.mvd_launch_count()
        mvd.mvd_deconvolve_planes(ctx, d, e)
        torch.cuda.synchronize()
        assert mvd.mvd_launch_count() - n0 == 1 + 2 * 4      # means + two kernels per iteration
        st = mvd.lib().mvd_deconvolve_planes(ctx.handle, None, 1, None, 3, 1, None)
        assert st == mvd.MVD_ERR_ARG
        assert mvd.mvd_last_error() != ""
        with pytest.raises(ValueError):
            mvd.mvd_deconvolve_planes(ctx, torch.ones((2, 3, 21, 30), device=DEV), e)
    finally:
        ctx.close()


def test_volume_1024_cubed_four_views_sampled_planes(mvd):
    """Four views of 1024^3 uint16 blobs (density 5e-5) at 0/90/180/270
    degrees with 41x41 PSFs sigma (1.8, 10), resliced on the GPU, 10
    iterations in sequential order over all 1024 planes; sampled planes
    against the FP64 oracle."""
    stacks, psfs = synth.volume_stacks(1024, 1024, 1024, 41, 10.0, 1.8, (0, 90, 180, 270), 5e-5, seed=0,
                                       device=DEV)
    V, Z, Y, X = stacks.shape
    ctx = mvd.mvd_create(V, psfs, 41, Z, X, 10, "zero", 1e-6)
    try:
        mvd.mvd_set_update_order(ctx, "sequential")
        assert mvd.mvd_get_info(ctx).algo == mvd.ALGO["fused"]
        planes = torch.empty((V, Y, Z, X), dtype=stacks.dtype, device=DEV)
        mvd.mvd_reslice(ctx, stacks, planes)
        sample = [3, 700]
        # the oracle's planes are cut from the synthetic stacks by torch
        # slicing (plane y of view v is stacks[v, :, y, :]), not taken from
        # the library's reslice
        phi = np.stack([stacks[:, :, i, :].to(torch.int32).cpu().numpy() for i in sample], axis=1)
        del stacks
        est = torch.empty((Y, Z, X), dtype=torch.float32, device=DEV)
        mvd.mvd_deconvolve_planes(ctx, planes, est)
        torch.cuda.synchronize()
        mvd.mvd_device_status(ctx)
    finally:
        ctx.close()
    ref = oracle.rl_planes(phi, psfs, 10, eps=1e-6, route="fft", order="sequential")
    assert_parity(est[sample].cpu().numpy(), ref, what="1024^3 4 views sampled planes")


def test_volume_512_cubed_two_views_sampled_planes(mvd):
    """The benchmarked workload in its launch configuration: 2 views of
    512^3 uint16 blobs (density 1e-4), 31x31 PSFs sigma (1.5, 8) turned by 90
    degrees, resliced on the GPU, 10 iterations over all 512 planes in one
    call; sampled planes against the FP64 oracle."""
    stacks, psfs = synth.volume_stacks(512, 512, 512, 31, 8.0, 1.5, (0, 90), 1e-4, seed=0, device=DEV)
    V, Z, Y, X = stacks.shape
    ctx = mvd.mvd_create(V, psfs, 31, Z, X, 10, "zero", 1e-6)
    try:
        planes = torch.empty((V, Y, Z, X), dtype=stacks.dtype, device=DEV)
        mvd.mvd_reslice(ctx, stacks, planes)
        est = torch.empty((Y, Z, X), dtype=torch.float32, device=DEV)
        mvd.mvd_deconvolve_planes(ctx, planes, est)
        torch.cuda.synchronize()
    finally:
        ctx.close()
    sample = [0, 255, 511]
    # oracle planes cut from the synthetic stacks (plane y of view v is
    # stacks[v, :, y, :]), plane by plane (uint16 CUDA tensors have no
    # advanced indexing)
    phi = np.stack([stacks[:, :, i, :].to(torch.int32).cpu().numpy() for i in sample], axis=1)
    ref = oracle.rl_planes(phi, psfs, 10, eps=1e-6, route="fft")
    assert_parity(est[sample].cpu().numpy(), ref, what="512^3 sampled planes")


def test_narrow_factors_of_large_psfs_run_with_21_central_taps(mvd):
    """41x41 PSFs sigma (1.8, 10) at 0/90 degrees: the lateral factors keep
    all but ~1e-7 of their mass in their 21 central taps (17 would leave
    ~2e-6, above the rank tolerance), so the fused kernels run those passes
    with 21 taps; the result matches the oracle."""
    c = synth.plane_case(seed=62, H=160, W=272, n_planes=2, n_blobs=60, K=41, sigma_axial=10.0,
                         sigma_lateral=1.8, angles=(0, 90, 180, 270), iters=5, dtype=np.uint16)
    V, P, H, W = c.phi.shape
    ctx = mvd.mvd_create(V, c.psfs, 41, H, W, 5, "zero", 1e-6)
    try:
        info = mvd.mvd_get_info(ctx)
        assert info.flops_blur == 2 * 2 * (41 + 21) and info.flops_corr == 4 * 2 * (41 + 21)
    finally:
        ctx.close()
    ref = oracle.rl_planes(c.phi, c.psfs, 5, eps=1e-6, route="fft", order="sequential")
    assert_parity(run_gpu(mvd, c.phi, c.psfs, 5, order="sequential"), ref, what="21-tap factors, 4 views")
    # two views with distinct PSFs: the simultaneous product (kernel B's
    # rank-1 path over both views)
    phi2, psfs2 = c.phi[:2], c.psfs[:2]
    ref = oracle.rl_planes(phi2, psfs2, 5, eps=1e-6, route="fft")
    assert_parity(run_gpu(mvd, phi2, psfs2, 5), ref, what="21-tap factors, 2 views")


def test_narrow_factors_run_with_central_taps(mvd):
    """31x31 PSFs sigma (1.5, 8) turned by 90 degrees: the lateral factors
    keep all but ~1e-8 of their mass in their 17 central taps, so the fused
    kernels run those passes short (info.flops_* count the taps run); the
    result still matches the oracle.  Weighted runs keep every tap (a
    zero-weight region's only signal comes through the tails): checked with
    weights through kernel B's general path."""
    c = synth.plane_case(seed=61, H=200, W=300, n_planes=2, n_blobs=80, K=31, sigma_axial=8.0,
                         sigma_lateral=1.5, iters=5, dtype=np.uint16)
    V, P, H, W = c.phi.shape
    ctx = mvd.mvd_create(V, c.psfs, 31, H, W, 5, "zero", 1e-6)
    try:
        info = mvd.mvd_get_info(ctx)
        assert info.flops_blur == 2 * 2 * (31 + 17) and info.flops_corr == 2 * 2 * (31 + 17)
        mvd.mvd_set_rank_tolerance(ctx, 0.0)          # exact factors (every term kept): no short passes
        info0 = mvd.mvd_get_info(ctx)
        assert info0.flops_blur == 2 * info0.blur_terms * 62
    finally:
        ctx.close()
    ref = oracle.rl_planes(c.phi, c.psfs, 5, eps=1e-6, route="fft")
    assert_parity(run_gpu(mvd, c.phi, c.psfs, 5), ref, what="short factors")
    w = np.random.default_rng(61).uniform(0.3, 1.0, size=c.phi.shape).astype(np.float32)
    ctx = mvd.mvd_create(V, c.psfs, 31, H, W, 5, "zero", 1e-6)
    try:
        wt = torch.from_numpy(w).to(DEV)
        mvd.mvd_set_weights(ctx, wt)
        assert mvd.mvd_get_info(ctx).flops_blur == 2 * 2 * 62
        d = torch.from_numpy(c.phi).to(DEV)
        est = torch.empty((P, H, W), device=DEV)
        mvd.mvd_deconvolve_planes(ctx, d, est)
        torch.cuda.synchronize()
        got = est.cpu().numpy()
    finally:
        ctx.close()
    refw = oracle.rl_planes(c.phi, c.psfs, 5, eps=1e-6, weights=w.astype(np.float64))
    assert_parity(got, refw, what="short factors, weighted")
