"""3D MV-RL route (views turned about the rotation axis: PSF a_v(y) P_v(z, x))
against the FP64 oracle, its reduction to the plane-wise method, and the
comparison the plane-wise approximation is judged by."""

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


def run(mvd, phi, psfs, axial, iters, boundary="zero", order="simultaneous"):
    V, P, H, W = phi.shape
    K = psfs.shape[-1]
    ctx = mvd.mvd_create(V, psfs, K, H, W, iters, boundary, 1e-6)
    try:
        mvd.mvd_set_update_order(ctx, order)
        mvd.mvd_set_axial_psfs(ctx, axial)
        d = torch.from_numpy(np.ascontiguousarray(phi)).to(DEV)
        est = torch.empty((P, H, W), device=DEV)
        mvd.mvd_deconvolve_planes(ctx, d, est)
        torch.cuda.synchronize()
        mvd.mvd_device_status(ctx)
        return est.cpu().numpy()
    finally:
        ctx.close()


@pytest.mark.parametrize("boundary", ["zero", "circular"])
@pytest.mark.parametrize("order", ["simultaneous", "sequential"])
def test_3d_route_matches_oracle(mvd, boundary, order):
    """2 views, 11x11 in-plane PSFs, axial profile sigma_y 2 (13 taps), 20
    planes of 70 x 136 (ragged tiles), uint16, 3 iterations."""
    c = synth.volume3d_case(20, 70, 136, 11, 3.0, 1.2, 2.0, n_blobs=40, seed=51)
    got = run(mvd, c["phi"], c["psfs"], c["axial"], 3, boundary, order)
    ref = oracle.rl3d(c["phi"], c["psfs"], c["axial"], 3, boundary=boundary, order=order)
    assert_parity(got, ref, what=f"3D {boundary} {order}")


def test_delta_profile_is_the_planewise_route(mvd):
    """A centred delta along the axis reproduces the plane-wise fused route
    bit for bit (same kernels, the axial passes copy)."""
    c = synth.volume3d_case(12, 64, 128, 15, 4.0, 1.5, 0.5, n_blobs=30, seed=52)
    delta = np.zeros((2, 5), dtype=np.float32)
    delta[:, 2] = 1.0
    got = run(mvd, c["phi"], c["psfs"], delta, 4)
    plane = run(mvd, c["phi"], c["psfs"], None, 4)
    np.testing.assert_array_equal(got, plane)


def test_3d_beats_planewise_on_axially_blurred_data(mvd):
    """Data blurred along the rotation axis (sigma_y 3): deconvolving in 3D
    gets closer to the truth than the plane-wise approximation, which
    ignores the axial blur (the comparison of Supp. Figs. 3-4)."""
    c = synth.volume3d_case(32, 96, 128, 21, 5.0, 1.5, 3.0, n_blobs=150, seed=53, noise=False)
    t = c["truth"]
    e3 = run(mvd, c["phi"], c["psfs"], c["axial"], 10)
    e2 = run(mvd, c["phi"], c["psfs"], None, 10)
    err3 = np.linalg.norm(e3 - t) / np.linalg.norm(t)
    err2 = np.linalg.norm(e2 - t) / np.linalg.norm(t)
    assert err3 < err2, (err3, err2)


def test_3d_errors(mvd):
    c = synth.volume3d_case(8, 32, 64, 7, 2.0, 1.0, 1.0, n_blobs=10, seed=54)
    V, P, H, W = c["phi"].shape
    ctx = mvd.mvd_create(V, c["psfs"], 7, H, W, 2, "zero", 1e-6)
    try:
        with pytest.raises(mvd.MvdError):
            mvd.mvd_set_axial_psfs(ctx, np.ones((V, 4), np.float32))     # even length
        with pytest.raises(mvd.MvdError):
            mvd.mvd_set_axial_psfs(ctx, -np.ones((V, 3), np.float32))    # negative
        mvd.mvd_set_axial_psfs(ctx, c["axial"])
        d = torch.from_numpy(c["phi"]).to(DEV)
        est = torch.empty((P, H, W), device=DEV)
        for algo in ("plain", "fft", "tensor"):
            mvd.mvd_set_algo(ctx, algo)
            with pytest.raises(mvd.MvdError) as e:
                mvd.mvd_deconvolve_planes(ctx, d, est)
            assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
        mvd.mvd_set_algo(ctx, "fused")
        with pytest.raises(mvd.MvdError) as e:
            mvd.mvd_deconvolve_planes(ctx, d, est, init_mean=False)
        assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
    finally:
        ctx.close()
