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
