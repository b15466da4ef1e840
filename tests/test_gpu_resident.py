"""Parity of the plane-resident route (MVD_ALGO_RESIDENT: one thread-block
cluster keeps a plane in shared memory for all iterations, neighbour rows
read through distributed shared memory) with the FP64 oracle, at the FP32
tolerances: the 128 x 128 two-view case, ragged planes (partial strips and
tiles) in both update orders, PSF sizes across the three size classes,
several SVD terms, a given first estimate, and 512 x 512 planes (16 CTAs per
cluster); planes that do not fit are refused."""

import numpy as np
import pytest

import oracle
from paper_1503_07998_gb300 import synth
from tests.parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mvd():
    from paper_1503_07998_gb300 import build as B
    B.build()
    from paper_1503_07998_gb300 import mvd as m
    m.lib()
    return m


def run_res(mvd, phi, psfs, iters, order="simultaneous", psi0=None):
    V, P, H, W = phi.shape
    ctx = mvd.mvd_create(V, psfs, psfs.shape[-1], H, W, iters, "zero", 1e-6)
    try:
        mvd.mvd_set_update_order(ctx, order)
        mvd.mvd_set_algo(ctx, "resident")
        d = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
        if psi0 is None:
            est = torch.empty((P, H, W), device="cuda")
        else:
            est = torch.from_numpy(np.ascontiguousarray(psi0, dtype=np.float32)).cuda()
        mvd.mvd_profile_enable(ctx, True)
        mvd.mvd_deconvolve_planes(ctx, d, est, init_mean=psi0 is None)
        torch.cuda.synchronize()
        assert "resident" in mvd.mvd_profile_read(ctx)
        return est.cpu().numpy()
    finally:
        ctx.close()


def test_one_128_plane_two_views_k17(mvd):
    c = synth.plane_case(seed=0)
    ref = oracle.rl_planes(c.phi, c.psfs, c.iters, eps=c.eps, route="fft")
    assert_parity(run_res(mvd, c.phi, c.psfs, c.iters), ref, what="resident 128^2")


@pytest.mark.parametrize("order", ["simultaneous", "sequential"])
@pytest.mark.parametrize("K", [5, 17, 31, 41])
def test_ragged_planes_every_size_class(mvd, order, K):
    """Planes of 150 x 200: the last strip is partial (150 = 4 x 32 + 22) and
    the last 16-column items run past the plane; uint16 data."""
    sa = max(1.0, K / 5.0)
    c = synth.plane_case(seed=40 + K, H=150, W=200, n_planes=3, n_blobs=80, K=K, sigma_axial=sa,
                         sigma_lateral=min(1.8, sa), iters=4, dtype=np.uint16)
    ref = oracle.rl_planes(c.phi, c.psfs, 4, eps=1e-6, route="fft", order=order)
    assert_parity(run_res(mvd, c.phi, c.psfs, 4, order=order), ref, what=f"resident K={K} {order}")


def test_oblique_views_several_terms(mvd):
    """Views at 0/45 degrees: the turned PSF has several SVD terms."""
    c = synth.plane_case(seed=60, H=96, W=112, n_planes=2, n_blobs=40, K=15, sigma_axial=4.0,
                         sigma_lateral=1.3, angles=(0, 45), iters=3, dtype=np.float32)
    ref = oracle.rl_planes(c.phi, c.psfs, 3, eps=1e-6, route="fft")
    assert_parity(run_res(mvd, c.phi, c.psfs, 3), ref, what="resident oblique")


def test_given_first_estimate(mvd):
    c = synth.plane_case(seed=61, H=70, W=90, n_planes=2, n_blobs=30, K=13, sigma_axial=3.0,
                         sigma_lateral=1.2, iters=3, dtype=np.float32)
    psi0 = np.random.default_rng(61).uniform(20, 60, size=(2, 70, 90))
    ref = oracle.rl_planes(c.phi, c.psfs, 3, eps=1e-6, psi0=psi0, route="fft")
    assert_parity(run_res(mvd, c.phi, c.psfs, 3, psi0=psi0), ref, what="resident psi0")


def test_512_planes_sixteen_ctas(mvd):
    """Two 512 x 512 planes, 31 x 31 PSFs sigma (1.5, 8) turned by 90
    degrees, 10 iterations: the 512^3 workload's planes, one cluster of 16
    CTAs per plane."""
    c = synth.plane_case(seed=62, H=512, W=512, n_planes=2, n_blobs=400, K=31, sigma_axial=8.0,
                         sigma_lateral=1.5, iters=10, dtype=np.uint16)
    ref = oracle.rl_planes(c.phi, c.psfs, 10, eps=1e-6, route="fft")
    assert_parity(run_res(mvd, c.phi, c.psfs, 10), ref, what="resident 512^2")


def test_planes_that_do_not_fit_are_refused(mvd):
    psfs = np.ones((2, 9, 9), np.float32) / 81
    for H, W in ((600, 600), (64, 520)):
        ctx = mvd.mvd_create(2, psfs, 9, H, W, 2, "zero", 1e-6)
        try:
            with pytest.raises(mvd.MvdError) as ei:
                mvd.mvd_set_algo(ctx, "resident")
            assert ei.value.status == mvd.MVD_ERR_UNSUPPORTED
        finally:
            ctx.close()
    ctx = mvd.mvd_create(2, psfs, 9, 64, 64, 2, "circular", 1e-6)
    try:
        with pytest.raises(mvd.MvdError):
            mvd.mvd_set_algo(ctx, "resident")
    finally:
        ctx.close()
