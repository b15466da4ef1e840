"""Parity of the MV-RL variants (Supp. Note 2 sec. 1) with the oracle on every
route: the library builds X_v on the host, factorises it, and the kernels
correlate with it in place of the flipped PSF."""

import numpy as np
import pytest

import oracle
from paper_1503_07998_gb300 import synth
from tests.parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
VARIANTS = ["efficient_bayesian", "optimization_1", "optimization_2"]


@pytest.fixture(scope="module")
def mvd():
    from paper_1503_07998_gb300 import build as B
    B.build()
    from paper_1503_07998_gb300 import mvd as m
    m.lib()
    return m


def run(mvd, case, variant, algo, order):
    V, P, H, W = case.phi.shape
    K = case.psfs.shape[-1]
    ctx = mvd.mvd_create(V, case.psfs, K, H, W, case.iters, case.boundary, case.eps)
    try:
        mvd.mvd_set_variant(ctx, variant)
        mvd.mvd_set_algo(ctx, algo)
        mvd.mvd_set_update_order(ctx, order)
        d = torch.from_numpy(np.ascontiguousarray(case.phi)).to(DEV)
        est = torch.empty((P, H, W), dtype=torch.float32, device=DEV)
        mvd.mvd_deconvolve_planes(ctx, d, est)
        torch.cuda.synchronize()
        mvd.mvd_device_status(ctx)
        return est.cpu().numpy(), mvd.mvd_get_info(ctx)
    finally:
        ctx.close()


def oracle_of(case, variant, order):
    X = oracle.correlation_kernels(case.psfs.astype(np.float64), variant)
    return oracle.rl_planes(case.phi, case.psfs, case.iters, boundary=case.boundary, eps=case.eps, order=order,
                            corr_kernels=X)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("algo", ["fused", "plain", "direct", "fft"])
def test_oblique_views_every_route(mvd, variant, algo):
    """Three views at 0/60/120 degrees (oblique PSFs: several SVD terms in
    both the blur and the correlation), two planes spanning several tiles
    with ragged edges, sequential order."""
    case = synth.plane_case(seed=31, H=72, W=150, n_planes=2, n_blobs=60, K=11, sigma_axial=3.0,
                            sigma_lateral=1.2, angles=(0.0, 60.0, 120.0), iters=3)
    got, info = run(mvd, case, variant, algo, "sequential")
    assert info.variant == mvd.VARIANT[variant]
    assert all(info.corr_rank[v] >= 1 for v in range(3))
    assert_parity(got, oracle_of(case, variant, "sequential"), what=f"{variant}/{algo}")


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("boundary", ["zero", "circular"])
def test_axis_aligned_views_rank_one_correlation(mvd, variant, boundary):
    """Two orthogonal axis-aligned Gaussian views: every X_v is separable, so
    the correlation runs on the rank-1 fast path; simultaneous order."""
    case = synth.plane_case(seed=32, H=96, W=136, n_planes=3, n_blobs=80, K=17, iters=4, boundary=boundary)
    got, info = run(mvd, case, variant, "fused", "simultaneous")
    assert list(info.corr_rank[:2]) == [1, 1]
    assert_parity(got, oracle_of(case, variant, "simultaneous"), what=f"{variant}/{boundary}")


def test_variant_switch_and_psf_update(mvd):
    """Switching the variant back to independent restores plain MV-RL
    bit for bit; mvd_set_psfs rebuilds the variant's kernels."""
    case = synth.plane_case(seed=33, H=64, W=130, n_planes=1, n_blobs=40, K=9, sigma_axial=2.5,
                            angles=(0.0, 90.0, 45.0), iters=2)
    V, P, H, W = case.phi.shape
    ctx = mvd.mvd_create(V, case.psfs, 9, H, W, case.iters, "zero", case.eps)
    try:
        mvd.mvd_set_update_order(ctx, "sequential")
        d = torch.from_numpy(np.ascontiguousarray(case.phi)).to(DEV)
        est = torch.empty((P, H, W), device=DEV)

        def go():
            mvd.mvd_deconvolve_planes(ctx, d, est)
            torch.cuda.synchronize()
            return est.cpu().numpy().copy()

        plain = go()
        mvd.mvd_set_variant(ctx, "optimization_2")
        v2 = go()
        assert not np.array_equal(plain, v2)
        mvd.mvd_set_variant(ctx, "independent")
        np.testing.assert_array_equal(go(), plain)
        other = synth.plane_case(seed=34, K=9, sigma_axial=4.0, sigma_lateral=1.0, angles=(30.0, 120.0, 75.0)).psfs
        mvd.mvd_set_variant(ctx, "efficient_bayesian")
        mvd.mvd_set_psfs(ctx, other)
        got = go()
        X = oracle.correlation_kernels(other.astype(np.float64), "efficient_bayesian")
        want = oracle.rl_planes(case.phi, other, case.iters, eps=case.eps, order="sequential", corr_kernels=X)
        assert_parity(got, want, what="after set_psfs")
        with pytest.raises(mvd.MvdError) as e:
            mvd.mvd_psf_grad(ctx, d)
        assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
    finally:
        ctx.close()


def test_batch_with_variant_volumes(mvd):
    """A batch mixing variants equals single contexts of the same variant."""
    vols = synth.uneven_volumes(3, seed=35, side=(40, 90), planes=(2, 4), views=(2, 3), psf=(5, 11),
                                iters=(2, 3), density=2e-3, device="cuda")
    names = ["optimization_1", "independent", "efficient_bayesian"]
    ests = [torch.empty((v["P"], v["H"], v["W"]), device="cuda") for v in vols]
    batch = mvd.mvd_batch_create([{"stacks": v["stacks"], "psfs": v["psfs"], "iters": v["iters"], "estimate": e,
                                   "variant": n} for v, e, n in zip(vols, ests, names)], order="sequential")
    try:
        mvd.mvd_batch_run(batch)
        torch.cuda.synchronize()
        for v, e, n in zip(vols, ests, names):
            V, H, P, W = v["stacks"].shape
            ctx = mvd.mvd_create(V, v["psfs"], v["K"], H, W, v["iters"], "zero", 1e-6)
            try:
                mvd.mvd_set_update_order(ctx, "sequential")
                mvd.mvd_set_variant(ctx, n)
                planes = torch.empty((V, P, H, W), dtype=v["stacks"].dtype, device="cuda")
                mvd.mvd_reslice(ctx, v["stacks"], planes)
                want = torch.empty((P, H, W), device="cuda")
                mvd.mvd_deconvolve_planes(ctx, planes, want)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(e.cpu().numpy(), want.cpu().numpy())
            finally:
                ctx.close()
    finally:
        batch.close()
