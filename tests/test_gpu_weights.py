"""Weighted MV-RL (per-pixel view weights, EM footprint normaliser) and the
padded-domain estimate on the GPU, against the FP64 oracle."""

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


def random_weights(rng, shape, K):
    """Weights in [0.2, 1] with a zero block per view wider than the PSF, so
    that the normaliser's floor (factor 1) is reached inside the plane."""
    w = rng.uniform(0.2, 1.0, size=shape)
    V, P, H, W = shape
    for v in range(V):
        y0 = rng.integers(0, max(1, H - 2 * K))
        x0 = rng.integers(0, max(1, W - 2 * K))
        w[v, :, y0:y0 + 2 * K, x0:x0 + 2 * K] = 0.0
    return w


def run(mvd, phi, psfs, w, iters, boundary="zero", algo="fused", order="simultaneous", variant=None):
    V, P, H, W = phi.shape
    K = psfs.shape[-1]
    ctx = mvd.mvd_create(V, psfs, K, H, W, iters, boundary, 1e-6)
    try:
        if variant:
            mvd.mvd_set_variant(ctx, variant)
        mvd.mvd_set_algo(ctx, algo)
        mvd.mvd_set_update_order(ctx, order)
        wt = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).to(DEV)
        mvd.mvd_set_weights(ctx, wt)
        d = torch.from_numpy(np.ascontiguousarray(phi)).to(DEV)
        est = torch.empty((P, H, W), device=DEV)
        mvd.mvd_deconvolve_planes(ctx, d, est)
        torch.cuda.synchronize()
        mvd.mvd_device_status(ctx)
        return est.cpu().numpy()
    finally:
        ctx.close()


@pytest.mark.parametrize("boundary", ["zero", "circular"])
@pytest.mark.parametrize("algo", ["fused", "plain", "direct"])
@pytest.mark.parametrize("order", ["simultaneous", "sequential"])
def test_random_weights_two_views(mvd, boundary, algo, order):
    """2 views, 17x17 Gaussians turned by 90 degrees, 3 planes of 130x260
    (several tiles, ragged), uint16 data, random weights with zero blocks."""
    c = synth.plane_case(seed=41, H=130, W=260, n_planes=3, n_blobs=80, K=17, iters=4, dtype=np.uint16,
                         boundary=boundary)
    rng = np.random.default_rng(41)
    w = random_weights(rng, c.phi.shape, 17)
    w32 = w.astype(np.float32).astype(np.float64)   # the GPU reads FP32 weights
    ref = oracle.rl_planes(c.phi, c.psfs, 4, boundary=boundary, eps=1e-6, order=order, weights=w32)
    got = run(mvd, c.phi, c.psfs, w, 4, boundary, algo, order)
    assert_parity(got, ref, what=f"weights {algo} {order} {boundary}")


def test_oblique_views_several_terms_and_variant(mvd):
    """3 views at 0/60/120 degrees (several SVD terms), FP32 data, ragged
    plane; plain MV-RL and the efficient Bayesian variant."""
    c = synth.plane_case(seed=42, H=97, W=141, n_planes=2, n_blobs=50, K=11, sigma_axial=3.0,
                         sigma_lateral=1.2, angles=(0.0, 60.0, 120.0), iters=3)
    rng = np.random.default_rng(42)
    w = random_weights(rng, c.phi.shape, 11).astype(np.float32).astype(np.float64)
    ref = oracle.rl_planes(c.phi, c.psfs, 3, eps=1e-6, order="sequential", weights=w)
    assert_parity(run(mvd, c.phi, c.psfs, w, 3, order="sequential"), ref, what="weights oblique")
    X = oracle.correlation_kernels(c.psfs.astype(np.float64), "efficient_bayesian")
    ref = oracle.rl_planes(c.phi, c.psfs, 3, eps=1e-6, order="sequential", weights=w, corr_kernels=X)
    assert_parity(run(mvd, c.phi, c.psfs, w, 3, order="sequential", variant="efficient_bayesian"), ref,
                  what="weights variant")


def test_unit_weights_equal_unweighted_circular(mvd):
    c = synth.plane_case(seed=43, H=128, W=256, n_planes=2, n_blobs=60, K=15, iters=3, boundary="circular")
    ones = np.ones(c.phi.shape)
    got = run(mvd, c.phi, c.psfs, ones, 3, "circular")
    ref = oracle.rl_planes(c.phi, c.psfs, 3, boundary="circular", eps=1e-6)
    assert_parity(got, ref, what="unit weights")


@pytest.mark.parametrize("dtype,per_plane,R", [(np.uint16, False, 15), (np.float32, True, 15), (np.uint16, False, 16)])
def test_padded_domain_pipeline(mvd, dtype, per_plane, R):
    """Planes embedded on the GPU into the data + PSF padded domain (zero
    weights in the padding; one weight plane per view shared by all planes,
    or one per plane), deconvolved there, cropped back; the embedding is
    bit-exact and the estimate matches the oracle's padded-domain RL.  R = 16
    pads 200 to a 16-multiple width (TMA and vector loads)."""
    K = 31
    c = synth.plane_case(seed=44, H=96, W=200, n_planes=2, n_blobs=60, K=K, sigma_axial=8.0, iters=5,
                         dtype=dtype)
    V, P, H, W = c.phi.shape
    d = torch.from_numpy(np.ascontiguousarray(c.phi)).to(DEV)
    pd, w = mvd.mvd_embed_padded(d, R, per_plane_weights=per_plane)
    want_pd, want_w = oracle.embed_padded(c.phi, R)
    np.testing.assert_array_equal(pd.cpu().numpy(), want_pd)
    assert w.shape[1] == (P if per_plane else 1)
    np.testing.assert_array_equal(w.cpu().numpy(), want_w[:, :w.shape[1]].astype(np.float32))
    ctx = mvd.mvd_create(V, c.psfs, K, H + 2 * R, W + 2 * R, 5, "zero", 1e-6)
    try:
        mvd.mvd_set_weights(ctx, w)
        est = torch.empty((P, H + 2 * R, W + 2 * R), device=DEV)
        mvd.mvd_deconvolve_planes(ctx, pd, est)
        crop = mvd.mvd_crop_planes(est, R)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(crop.cpu().numpy(), oracle.crop_padded(est.cpu().numpy(), R))
    finally:
        ctx.close()
    ref = oracle.rl_planes(want_pd, c.psfs, 5, eps=1e-6, weights=want_w)
    assert_parity(est.cpu().numpy(), ref, what=f"padded domain {np.dtype(dtype).name}")


def test_weight_errors(mvd):
    c = synth.plane_case(seed=45, H=64, W=128, n_planes=2, n_blobs=20, K=9, iters=2)
    V, P, H, W = c.phi.shape
    ctx = mvd.mvd_create(V, c.psfs, 9, H, W, 2, "zero", 1e-6)
    try:
        w = torch.ones((V, P, H, W), device=DEV)
        mvd.mvd_set_weights(ctx, w)
        d = torch.from_numpy(c.phi).to(DEV)
        est = torch.empty((P, H, W), device=DEV)
        with pytest.raises(mvd.MvdError) as e:
            mvd.mvd_deconvolve_planes(ctx, d[:, :1].contiguous(), est[:1])
        assert e.value.status == mvd.MVD_ERR_ARG
        for algo in ("fft", "tensor"):
            mvd.mvd_set_algo(ctx, algo)
            with pytest.raises(mvd.MvdError) as e:
                mvd.mvd_deconvolve_planes(ctx, d, est)
            assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
        mvd.mvd_set_algo(ctx, "fused")
        with pytest.raises(mvd.MvdError) as e:
            mvd.mvd_psf_grad(ctx, d)
        assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
        assert mvd.mvd_autotune(ctx, d) == "fused"      # the Fourier route takes no weights
        mvd.mvd_set_weights(ctx, None)                   # cleared: plain MV-RL again
        mvd.mvd_deconvolve_planes(ctx, d, est)
        torch.cuda.synchronize()
        ref = oracle.rl_planes(c.phi, c.psfs, 2, eps=1e-6)
        assert_parity(est.cpu().numpy(), ref, what="weights cleared")
    finally:
        ctx.close()
