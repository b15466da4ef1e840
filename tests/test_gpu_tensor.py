"""Parity of the optional tensor-core route (MVD_ALGO_TENSOR: BF16x3 tcgen05
passes, FP32 ratio/update) with the FP64 oracle, at the same tolerances as
the FP32 routes.  Each case records its measured error; with MVD_PARITY_LOG
naming a file the errors are appended there (one line per case)."""

import json
import os

import numpy as np
import pytest

import oracle
from paper_1503_07998_gb300 import synth
from tests.parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def mvd():
    from paper_1503_07998_gb300 import build as B
    B.build()
    from paper_1503_07998_gb300 import mvd as m
    m.lib()
    return m


def check(got, ref, what, rel_l2=None):
    r, p, raw = assert_parity(got, ref, what=what) if rel_l2 is None else assert_parity(got, ref, rel_l2, what=what)
    path = os.environ.get("MVD_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": what, "rel_l2": r, "per_pixel": p, "raw_max": raw}) + "\n")


def run_tc(mvd, phi, psfs, iters, boundary="zero", eps=1e-6, order="simultaneous", variant=None):
    V, P, H, W = phi.shape
    K = psfs.shape[-1]
    ctx = mvd.mvd_create(V, psfs, K, H, W, iters, boundary, eps)
    try:
        if variant:
            mvd.mvd_set_variant(ctx, variant)
        mvd.mvd_set_algo(ctx, "tensor")
        mvd.mvd_set_update_order(ctx, order)
        info = mvd.mvd_get_info(ctx)
        assert info.algo == mvd.ALGO["tensor"] and info.tile_w == 128
        d = torch.from_numpy(np.ascontiguousarray(phi)).to(DEV)
        est = torch.empty((P, H, W), dtype=torch.float32, device=DEV)
        mvd.mvd_profile_enable(ctx, True)
        mvd.mvd_deconvolve_planes(ctx, d, est)
        torch.cuda.synchronize()
        mvd.mvd_device_status(ctx)
        prof = mvd.mvd_profile_read(ctx)
        if iters > 0:
            # launches whose views share one rank-1 factorisation run on the
            # warp-specialised kernels (tcw_*), the others on tc_*
            assert any(k in prof for k in ("tc_blur_ratio", "tcw_blur_ratio"))
            assert any(k in prof for k in ("tc_correlate_update", "tcw_correlate_update"))
        return est.cpu().numpy()
    finally:
        ctx.close()


@pytest.mark.parametrize("name", ["small_zero", "small_circular"])
def test_golden_fixtures(mvd, name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        case = json.load(f)
    phi = np.array(case["phi"], dtype=np.float32)
    psf = np.array(case["psf"], dtype=np.float32)
    got = run_tc(mvd, phi, psf, case["iters"], case["boundary"], case["eps"])
    check(got, np.array(case["expected"]), f"tensor golden {name}")


def test_single_plane_two_views_k17(mvd):
    """One 128x128 FP32 plane, 2 views, 17x17 sigma (1.5, 6) PSFs turned by
    90 degrees, 200 blobs, seed 0, 10 iterations."""
    c = synth.plane_case(seed=0)
    ref = oracle.rl_planes(c.phi, c.psfs, c.iters, boundary="zero", eps=c.eps, route="fft")
    check(run_tc(mvd, c.phi, c.psfs, c.iters), ref, "tensor 128^2 K=17 2 views 10 it")


@pytest.mark.parametrize("boundary", ["zero", "circular"])
@pytest.mark.parametrize("K,V,H,W,dtype", [
    (1, 1, 33, 47, np.float32),
    (3, 3, 70, 150, np.uint16),
    (17, 2, 130, 260, np.uint16),
    (31, 2, 97, 141, np.float32),
    (33, 2, 200, 136, np.float32),
    (41, 4, 150, 136, np.uint16),
    (47, 1, 64, 256, np.float32),
])
def test_ragged_tiles_general_psfs(mvd, boundary, K, V, H, W, dtype):
    """Random non-symmetric PSFs (every SVD term kept, so K terms per view
    accumulate in one tensor-memory accumulator), several tiles, ragged
    edges; widths that are multiples of 4 take TMA tile loads, the others the
    software loader."""
    if boundary == "circular" and K > min(H, W):
        pytest.skip("circular needs K <= plane")
    rng = np.random.default_rng(K * 1000 + V)
    psfs = (rng.random((V, K, K)) + 0.05).astype(np.float32)
    psfs /= psfs.sum(axis=(1, 2), keepdims=True)
    P = 2
    base = rng.uniform(20, 400, size=(V, P, H, W))
    phi = base.astype(dtype) if dtype == np.float32 else np.round(base).astype(np.uint16)
    ref = oracle.rl_planes(phi, psfs, 3, boundary=boundary, eps=1e-6, route="fft")
    # BF16x3 keeps about 2^-16 of each product; a random PSF's SVD terms have
    # mixed signs and cancel, so the error of their sum is relative to the
    # terms, not to the result.  With 41 such terms per view and four views
    # multiplied in the simultaneous product the stated bound of this route
    # is rel-L2 3e-4 (measured 2.0e-4); every other case meets the FP32
    # tolerances.
    rel = 3e-4 if (K >= 41 and V >= 4) else None
    check(run_tc(mvd, phi, psfs, 3, boundary), ref, f"tensor K={K} V={V} {H}x{W} {boundary}", rel)


@pytest.mark.parametrize("boundary", ["zero", "circular"])
def test_four_views_sequential_k41(mvd, boundary):
    """Views at 0/90/180/270 degrees, 41x41 sigma (1.8, 10), 10 iterations in
    sequential order (the precision configuration's PSFs and order)."""
    c = synth.plane_case(seed=3, H=200, W=168, n_planes=3, n_blobs=40, K=41, sigma_axial=10.0,
                         sigma_lateral=1.8, angles=(0, 90, 180, 270), dtype=np.uint16)
    ref = oracle.rl_planes(c.phi, c.psfs, 10, boundary=boundary, eps=1e-6, route="fft", order="sequential")
    check(run_tc(mvd, c.phi, c.psfs, 10, boundary, order="sequential"), ref,
          f"tensor 4 views K=41 sequential {boundary}")


@pytest.mark.parametrize("variant", ["efficient_bayesian", "optimization_2"])
def test_variants_oblique(mvd, variant):
    c = synth.plane_case(seed=31, H=72, W=152, n_planes=2, n_blobs=60, K=11, sigma_axial=3.0,
                         sigma_lateral=1.2, angles=(0.0, 60.0, 120.0), iters=3)
    X = oracle.correlation_kernels(c.psfs.astype(np.float64), variant)
    ref = oracle.rl_planes(c.phi, c.psfs, 3, eps=c.eps, order="sequential", corr_kernels=X)
    check(run_tc(mvd, c.phi, c.psfs, 3, order="sequential", variant=variant), ref, f"tensor variant {variant}")


def test_first_iteration_from_given_estimate(mvd):
    """psi0 given (TMA path from the first iteration on)."""
    c = synth.plane_case(seed=5, H=96, W=256, n_planes=2, n_blobs=50, K=15)
    rng = np.random.default_rng(5)
    psi0 = rng.uniform(50, 150, size=(2, 96, 256)).astype(np.float32)
    V, P, H, W = c.phi.shape
    ctx = mvd.mvd_create(V, c.psfs, 15, H, W, 4, "zero", 1e-6)
    try:
        mvd.mvd_set_algo(ctx, "tensor")
        d = torch.from_numpy(c.phi).to(DEV)
        est = torch.from_numpy(psi0).to(DEV)
        mvd.mvd_deconvolve_planes(ctx, d, est, init_mean=False)
        torch.cuda.synchronize()
        got = est.cpu().numpy()
    finally:
        ctx.close()
    ref = oracle.rl_planes(c.phi, c.psfs, 4, eps=1e-6, psi0=psi0)
    check(got, ref, "tensor psi0 given")


def _volume(mvd, n, K, sigma_axial, sigma_lateral, angles, density, order, sample):
    stacks, psfs = synth.volume_stacks(n, n, n, K, sigma_axial, sigma_lateral, angles, density, seed=0, device=DEV)
    V, Z, Y, X = stacks.shape
    ctx = mvd.mvd_create(V, psfs, K, Z, X, 10, "zero", 1e-6)
    try:
        mvd.mvd_set_update_order(ctx, order)
        mvd.mvd_set_algo(ctx, "tensor")
        planes = torch.empty((V, Y, Z, X), dtype=stacks.dtype, device=DEV)
        mvd.mvd_reslice(ctx, stacks, planes)
        del stacks
        est = torch.empty((Y, Z, X), dtype=torch.float32, device=DEV)
        mvd.mvd_deconvolve_planes(ctx, planes, est)
        torch.cuda.synchronize()
        mvd.mvd_device_status(ctx)
    finally:
        ctx.close()
    phi = np.stack([planes[:, i].cpu().numpy() for i in sample], axis=1)
    ref = oracle.rl_planes(phi, psfs, 10, eps=1e-6, route="fft", order=order)
    return est[sample].cpu().numpy(), ref


def test_volume_512_cubed_two_views_sampled_planes(mvd):
    """The benchmarked workload (2 views, 512^3, K=31) on the tensor route."""
    got, ref = _volume(mvd, 512, 31, 8.0, 1.5, (0, 90), 1e-4, "simultaneous", [0, 255, 511])
    check(got, ref, "tensor 512^3 2 views K=31 sampled planes")


def test_volume_1024_cubed_four_views_sampled_planes(mvd):
    """The precision configuration: 4 views of 1024^3 at 0/90/180/270 degrees,
    41x41 PSFs sigma (1.8, 10), 10 iterations, tensor route."""
    got, ref = _volume(mvd, 1024, 41, 10.0, 1.8, (0, 90, 180, 270), 5e-5, "sequential", [3, 700])
    check(got, ref, "tensor 1024^3 4 views K=41 sampled planes")
