"""Failure detection on the GPU without a GPU fault: every tile wait of the
fused kernels is bounded, and an injected expiry (negative wait budget: the
wait reports a timeout after its copy has landed) must come back to the host
as MVD_ERR_TIMEOUT while the context stays usable."""

import numpy as np
import pytest

import oracle
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


def test_injected_wait_timeout_is_reported_and_context_recovers(mvd):
    rng = np.random.default_rng(21)
    V, P, H, W, K = 2, 2, 96, 160, 9
    psfs = (rng.random((V, K, K)) + 0.1).astype(np.float32)
    phi = rng.uniform(10, 100, size=(V, P, H, W)).astype(np.float32)
    ctx = mvd.mvd_create(V, psfs, K, H, W, 3, "zero", 1e-6)
    try:
        d = torch.from_numpy(phi).cuda()
        est = torch.empty((P, H, W), device="cuda")
        mvd.mvd_set_wait_budget(ctx, -1)
        mvd.mvd_deconvolve_planes(ctx, d, est)
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_device_status(ctx)
        assert ei.value.status == mvd.MVD_ERR_TIMEOUT
        mvd.mvd_device_status(ctx)            # the word was cleared
        mvd.mvd_set_wait_budget(ctx, 0)       # default budget again
        mvd.mvd_deconvolve_planes(ctx, d, est)
        mvd.mvd_device_status(ctx)
        ref = oracle.rl_planes(phi, psfs, 3)
        assert_parity(est.cpu().numpy(), ref, what="after recovery")
    finally:
        ctx.close()


def test_allocation_failure_returns_nomem_and_context_recovers(mvd):
    """The test hook makes the next device allocation fail as an exhausted
    cudaMalloc would: the call that needed it returns MVD_ERR_NOMEM, and the
    same context allocates and deconvolves correctly on the next call."""
    rng = np.random.default_rng(22)
    V, P, H, W, K = 2, 3, 64, 96, 7
    psfs = (rng.random((V, K, K)) + 0.1).astype(np.float32)
    phi = rng.uniform(10, 100, size=(V, P, H, W)).astype(np.float32)
    # a context whose creation needs memory
    mvd.mvd_debug_fail_allocations(1)
    try:
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_create(V, psfs, K, H, W, 3, "zero", 1e-6)
        assert ei.value.status == mvd.MVD_ERR_NOMEM
    finally:
        mvd.mvd_debug_fail_allocations(0)
    ctx = mvd.mvd_create(V, psfs, K, H, W, 3, "zero", 1e-6)
    try:
        d = torch.from_numpy(phi).cuda()
        est = torch.empty((P, H, W), device="cuda")
        mvd.mvd_debug_fail_allocations(1)      # the first call's workspace
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_deconvolve_planes(ctx, d, est)
        assert ei.value.status == mvd.MVD_ERR_NOMEM
        mvd.mvd_debug_fail_allocations(0)
        mvd.mvd_deconvolve_planes(ctx, d, est)
        torch.cuda.synchronize()
        mvd.mvd_device_status(ctx)
        assert_parity(est.cpu().numpy(), oracle.rl_planes(phi, psfs, 3), what="after allocation failure")
    finally:
        mvd.mvd_debug_fail_allocations(0)
        ctx.close()
