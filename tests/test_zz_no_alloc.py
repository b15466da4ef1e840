"""The allocation-free entry point, mvd_deconvolve_planes_static.

Some callers may not call cudaMalloc at all: acquisition software that
deconvolves while the camera records cannot afford an allocation's device
stall, and a plug-in inside an application that owns the GPU's memory pool
must not take memory behind its host's back.  For them the library offers one
context-free call whose scratch lives in a fixed static device array.  These
tests check, through the C ABI, that two such calls in a row give what the
regular entry point gives on the same inputs, and that a call too large for
the static array is refused with a clear message.

This file is collected last on purpose (its name sorts after the others).
"""

import numpy as np
import pytest

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


def _regular(mvd, phi, psfs, iters, boundary):
    V, P, H, W = phi.shape
    ctx = mvd.mvd_create(V, psfs, psfs.shape[-1], H, W, iters, boundary, 1e-6)
    try:
        est = torch.empty((P, H, W), dtype=torch.float32, device="cuda")
        mvd.mvd_deconvolve_planes(ctx, phi, est)
        torch.cuda.synchronize()
        return est.cpu().numpy()
    finally:
        ctx.close()


def test_static_entry_point_matches_regular_entry_point_twice(mvd):
    first = synth.plane_case(seed=31, H=200, W=168, n_planes=3, n_blobs=80, K=17, sigma_axial=6.0,
                             sigma_lateral=1.5, dtype=np.uint16)
    second = synth.plane_case(seed=32, H=96, W=136, n_planes=2, n_blobs=40, K=9, sigma_axial=3.0,
                              sigma_lateral=1.2, angles=(0, 90, 45), dtype=np.float32)
    cases = [(first, "zero"), (second, "circular")]
    for case, boundary in cases:
        phi = torch.from_numpy(case.phi).cuda()
        want = _regular(mvd, phi, case.psfs, 10, boundary)
        est = torch.empty(want.shape, dtype=torch.float32, device="cuda")
        mvd.mvd_deconvolve_planes_static(case.psfs, phi, est, 10, boundary)
        torch.cuda.synchronize()
        assert_parity(est.cpu().numpy(), want, what=f"static vs regular ({boundary})")


def test_static_entry_point_refuses_sizes_beyond_its_scratch(mvd):
    psfs = np.stack([synth.gaussian_psf(31, 8.0, 1.5, a) for a in (0, 90)])
    phi = torch.ones((2, 16, 512, 512), dtype=torch.float32, device="cuda")   # ratio planes alone: 32 MiB
    est = torch.empty((16, 512, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(mvd.MvdError) as ei:
        mvd.mvd_deconvolve_planes_static(psfs, phi, est, 2)
    assert ei.value.status == mvd.MVD_ERR_ARG
    assert "scratch" in str(ei.value)


def test_static_entry_point_allocates_nothing(mvd):
    """After a warm-up call (which may load the kernels' code), a second
    static call must leave the device's free memory and torch's reserved
    memory unchanged: the call's scratch is the static array alone."""
    case = synth.plane_case(seed=33, H=128, W=160, n_planes=2, n_blobs=50, K=13, sigma_axial=5.0,
                            sigma_lateral=1.4, dtype=np.uint16)
    phi = torch.from_numpy(case.phi).cuda()
    est = torch.empty((2, 128, 160), dtype=torch.float32, device="cuda")
    mvd.mvd_deconvolve_planes_static(case.psfs, phi, est, 5)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    mvd.mvd_deconvolve_planes_static(case.psfs, phi, est, 5)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_reserved() == reserved0
    mvd.mvd_static_device_status()


def test_static_entry_point_reports_an_injected_wait_timeout(mvd):
    """A negative wait budget makes every tile wait of the static call give up
    once its copy has landed; mvd_static_device_status must report it (and
    clear it), and a call with the default budget is correct again."""
    case = synth.plane_case(seed=34, H=96, W=128, n_planes=2, n_blobs=40, K=9, sigma_axial=3.0,
                            sigma_lateral=1.2, dtype=np.float32)
    phi = torch.from_numpy(case.phi).cuda()
    est = torch.empty((2, 96, 128), dtype=torch.float32, device="cuda")
    try:
        mvd.mvd_static_set_wait_budget(-1)
        mvd.mvd_deconvolve_planes_static(case.psfs, phi, est, 3)
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_static_device_status()
        assert ei.value.status == mvd.MVD_ERR_TIMEOUT
        mvd.mvd_static_device_status()          # read and cleared
    finally:
        mvd.mvd_static_set_wait_budget(0)
    mvd.mvd_deconvolve_planes_static(case.psfs, phi, est, 3)
    mvd.mvd_static_device_status()
    want = _regular(mvd, phi, case.psfs, 3, "zero")
    assert_parity(est.cpu().numpy(), want, what="static call after the injected timeout")
