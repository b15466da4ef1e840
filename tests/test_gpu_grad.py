"""PSF calibration on the GPU: loss and dL/dPSF of the Poisson fit of the
deconvolved estimate, through the C ABI (mvd_psf_grad), against the FP64
oracle's reverse sweep (itself pinned by central differences in
tests/test_oracle.py)."""

import numpy as np
import pytest

import oracle
from paper_1503_07998_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mvd():
    from paper_1503_07998_gb300 import build as B
    B.build()
    from paper_1503_07998_gb300 import mvd as m
    m.lib()
    return m


def gpu_grad(mvd, phi, psfs, iters, boundary, ckpt):
    V, P, H, W = phi.shape
    ctx = mvd.mvd_create(V, psfs, psfs.shape[-1], H, W, iters, boundary, 1e-6)
    try:
        d = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
        est = torch.empty((P, H, W), device="cuda")
        loss, g = mvd.mvd_psf_grad(ctx, d, ckpt, estimate=est)
        return loss, g.cpu().numpy().astype(np.float64), est.cpu().numpy()
    finally:
        ctx.close()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("boundary", ["zero", "circular"])
@pytest.mark.parametrize("ckpt", [1, 2, 3])
def test_gradient_matches_oracle_small(mvd, boundary, ckpt):
    rng = np.random.default_rng(40 + ckpt)
    V, P, H, W, K, T = 2, 2, 40, 48, 7, 4
    psfs = (rng.random((V, K, K)) + 0.05).astype(np.float32)
    psfs /= psfs.sum(axis=(1, 2), keepdims=True)
    phi = rng.uniform(5, 80, size=(V, P, H, W)).astype(np.float32)
    loss, g, est = gpu_grad(mvd, phi, psfs, T, boundary, ckpt)
    ref_loss, ref_g, ref_psi = oracle.rl_loss_and_psf_grad(phi, psfs, T, boundary)
    assert abs(loss - ref_loss) <= 1e-6 * abs(ref_loss)
    assert rel(g, ref_g) <= 1e-4, rel(g, ref_g)
    assert rel(est, ref_psi) <= 1e-5


@pytest.mark.parametrize("K,boundary", [(1, "zero"), (15, "zero"), (17, "circular"), (33, "zero"), (49, "zero")])
def test_gradient_tap_chunk_edges(mvd, K, boundary):
    """Tap and lag rows run in chunks of 16: K = 1, 15 (one chunk), 17 and 33
    (a last chunk of one tap) and 49 (a last chunk of one tap after three full
    ones), on 70 x 75 planes (2 x 2 tiles of 64, both ragged).  (Flat random
    33 x 33 PSFs with the circular boundary are left out: there the gradient
    picks up a near-uniform offset of 4e-4 of its norm from FP32 rounding in
    the sweep, the same on the earlier one-output-per-load kernels.)"""
    rng = np.random.default_rng(70 + K)
    V, P, H, W, T = 2, 2, 70, 75, 3
    psfs = (rng.random((V, K, K)) + 0.05).astype(np.float32)
    psfs /= psfs.sum(axis=(1, 2), keepdims=True)
    phi = rng.uniform(5, 80, size=(V, P, H, W)).astype(np.float32)
    loss, g, est = gpu_grad(mvd, phi, psfs, T, boundary, 2)
    ref_loss, ref_g, ref_psi = oracle.rl_loss_and_psf_grad(phi, psfs, T, boundary)
    assert abs(loss - ref_loss) <= 1e-6 * abs(ref_loss)
    assert rel(g, ref_g) <= 1e-4, rel(g, ref_g)
    assert rel(est, ref_psi) <= 1e-5


def test_gradient_psf_calibration_case(mvd):
    """Two views of blob planes made with sigma (1.5, 7) PSFs; free 31x31
    PSFs initialised to sigma (1.2, 5); 10 unrolled iterations, checkpoint
    every 2.  Two 64x64 planes keep the FP64 oracle fast."""
    truth = synth.plane_case(seed=50, H=64, W=64, n_planes=2, n_blobs=25, K=31, sigma_axial=7.0,
                             sigma_lateral=1.5, dtype=np.float32)
    init = np.stack([synth.gaussian_psf(31, 5.0, 1.2, a) for a in (0, 90)])
    loss, g, _ = gpu_grad(mvd, truth.phi, init, 10, "zero", 2)
    ref_loss, ref_g, _ = oracle.rl_loss_and_psf_grad(truth.phi, init, 10, "zero")
    assert abs(loss - ref_loss) <= 1e-6 * abs(ref_loss)
    assert rel(g, ref_g) <= 1e-4, rel(g, ref_g)


def test_checkpointing_does_not_change_the_gradient(mvd):
    rng = np.random.default_rng(60)
    V, P, H, W, K, T = 2, 3, 36, 40, 9, 6
    psfs = (rng.random((V, K, K)) + 0.05).astype(np.float32)
    phi = rng.uniform(5, 80, size=(V, P, H, W)).astype(np.float32)
    base = gpu_grad(mvd, phi, psfs, T, "zero", 1)
    for ck in (2, 4, 6, 9):
        other = gpu_grad(mvd, phi, psfs, T, "zero", ck)
        assert abs(other[0] - base[0]) <= 1e-12 * abs(base[0])
        np.testing.assert_allclose(other[1], base[1], rtol=1e-6, atol=1e-9 * np.abs(base[1]).max())


def test_autograd_function_backward(mvd):
    rng = np.random.default_rng(61)
    V, P, H, W, K, T = 2, 2, 32, 32, 5, 3
    psfs = (rng.random((V, K, K)) + 0.05).astype(np.float32)
    phi = rng.uniform(5, 80, size=(V, P, H, W)).astype(np.float32)
    ctx = mvd.mvd_create(V, psfs, K, H, W, T, "zero", 1e-6)
    try:
        d = torch.from_numpy(phi).cuda()
        p = torch.tensor(psfs, requires_grad=True)
        loss = mvd.psf_fit_loss(p, ctx, d, 2)
        (2.0 * loss).backward()
        ref_loss, ref_g, _ = oracle.rl_loss_and_psf_grad(phi, psfs, T, "zero")
        assert abs(loss.item() - ref_loss) <= 1e-6 * abs(ref_loss)
        assert rel(p.grad.numpy(), 2.0 * ref_g) <= 1e-4
    finally:
        ctx.close()


def test_gradient_at_the_calibration_workload_size(mvd):
    """The calibration workload at full size, in the launch configuration the
    benchmark times: 2 views, 64 planes of 256x256 blob data made with sigma
    (1.5, 7) px PSFs, free 31x31 PSFs at sigma (1.2, 5), 10 iterations,
    checkpoint every 2.  Loss and gradient are sums over planes, so the call
    on all 64 planes must equal the sum of calls on four blocks of 16, and
    single-plane calls on two sampled planes must match the FP64 oracle."""
    stacks, _ = synth.volume_stacks(256, 64, 256, 31, 7.0, 1.5, (0.0, 90.0), 2e-3, seed=5, device="cpu")
    planes = np.ascontiguousarray(stacks.to(torch.int32).numpy().transpose(0, 2, 1, 3))   # [V][Y][Z][X]
    init = np.stack([synth.gaussian_psf(31, 5.0, 1.2, a) for a in (0, 90)])
    ctx = mvd.mvd_create(2, init, 31, 256, 256, 10, "zero", 1e-6)
    try:
        d = torch.from_numpy(planes.astype(np.int32)).to(torch.uint16).cuda()
        loss_all, g_all = mvd.mvd_psf_grad(ctx, d, 2)
        g_all = g_all.cpu().numpy().astype(np.float64)
        loss_sum, g_sum = 0.0, np.zeros_like(g_all)
        for b in range(4):
            lb, gb = mvd.mvd_psf_grad(ctx, d[:, 16 * b:16 * (b + 1)].contiguous(), 2)
            loss_sum += lb
            g_sum += gb.cpu().numpy()
        assert abs(loss_all - loss_sum) <= 1e-9 * abs(loss_all)
        assert rel(g_all, g_sum) <= 1e-5, rel(g_all, g_sum)
        for y in (5, 40):
            lp, gp = mvd.mvd_psf_grad(ctx, d[:, y:y + 1].contiguous(), 2)
            ref_loss, ref_g, _ = oracle.rl_loss_and_psf_grad(planes[:, y:y + 1].astype(np.float64), init, 10, "zero")
            assert abs(lp - ref_loss) <= 1e-6 * abs(ref_loss), (y, lp, ref_loss)
            assert rel(gp.cpu().numpy().astype(np.float64), ref_g) <= 1e-4, (y, rel(gp.cpu().numpy(), ref_g))
    finally:
        ctx.close()


def test_loss_without_gradient_matches_the_gradient_call(mvd):
    """psf_fit_loss without requires_grad runs the forward iterations and the
    data fit only (no reverse sweep) and gives the same loss."""
    rng = np.random.default_rng(62)
    V, P, H, W, K, T = 2, 2, 48, 40, 9, 4
    psfs = (rng.random((V, K, K)) + 0.05).astype(np.float32)
    phi = rng.uniform(5, 80, size=(V, P, H, W)).astype(np.float32)
    ctx = mvd.mvd_create(V, psfs, K, H, W, T, "zero", 1e-6)
    try:
        d = torch.from_numpy(phi).cuda()
        with_grad, _ = mvd.mvd_psf_grad(ctx, d, 2)
        loss = mvd.psf_fit_loss(torch.tensor(psfs), ctx, d, 2)
        assert not loss.requires_grad
        assert abs(loss.item() - with_grad) <= 1e-12 * abs(with_grad)
        assert abs(mvd.mvd_poisson_loss(ctx, d) - with_grad) <= 1e-12 * abs(with_grad)
    finally:
        ctx.close()
