"""The persistent queue schedule of a batch (mvd_batch_set_schedule "queue"):
the fused-route volumes of each PSF-size class run as one launch over a
device-side queue of (phase, volume, plane, tile) items with per-plane
waits between phases.  Every volume is compared with the FP64 oracle on
sampled planes (and with the graph schedule), at toy sizes and on a seeded
subset of the 64-volume batch at its full plane sizes; an injected wait
timeout reaches the host as MVD_ERR_TIMEOUT and leaves the batch usable."""

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


def make_batch(mvd, vols, order, boundary="zero"):
    ests = [torch.full((v["P"], v["H"], v["W"]), -1.0, device="cuda") for v in vols]
    batch = mvd.mvd_batch_create([{"stacks": v["stacks"], "psfs": v["psfs"], "iters": v["iters"], "estimate": e}
                                  for v, e in zip(vols, ests)], boundary=boundary, order=order)
    return batch, ests


def planes_of(v):
    """[V][P][H][W] planes of a volume's [V][H][P][W] stacks (the oracle's reslice)."""
    return np.stack([oracle.reslice(s) for s in v["stacks"].cpu().numpy()])


def check_against_oracle(vols, ests, order, sample, boundary="zero"):
    for v, e in zip(vols, ests):
        got = e.cpu().numpy()
        planes = planes_of(v)
        for p in sample(v["P"]):
            phi = planes[:, p][:, None]
            ref = oracle.rl_planes(phi, v["psfs"], v["iters"], eps=1e-6, order=order, boundary=boundary, route="fft")
            assert_parity(got[p][None], ref, what=f"volume {v['H']}^2 x {v['P']} V={v['views']} K={v['K']} plane {p}")


@pytest.mark.parametrize("order", ["sequential", "simultaneous"])
def test_queue_schedule_small_uneven_volumes(mvd, order):
    """Nine volumes, two views at 0/90 degrees (rank-1 PSFs on the fused
    route) with PSF sides across the three size classes, and oblique ones
    that stay graph branches; two runs (the counters and the queue head are
    reset by the graph)."""
    vols = synth.uneven_volumes(9, seed=300, side=(40, 150), planes=(2, 7), views=(2, 3), psf=(5, 45),
                                iters=(2, 5), density=2e-3, device="cuda")
    batch, ests = make_batch(mvd, vols, order)
    try:
        mvd.mvd_batch_set_schedule(batch, "queue")
        mvd.mvd_batch_run(batch)
        mvd.mvd_batch_run(batch)
        mvd.mvd_batch_device_status(batch)
        info = mvd.mvd_batch_queue_info(batch)
        assert info["schedule"] == "queue"
        assert info["queue_volumes"] >= sum(v["views"] == 2 for v in vols)
        assert info["queue_items"] > 0
        queued = [e.clone() for e in ests]
        mvd.mvd_batch_set_schedule(batch, "graph")
        mvd.mvd_batch_run(batch)
        torch.cuda.synchronize()
        for q, g in zip(queued, ests):
            assert_parity(q.cpu().numpy(), g.cpu().numpy().astype(np.float64), what="queue vs graph schedule")
        check_against_oracle(vols, queued, order, lambda P: sorted({0, P // 2, P - 1}))
    finally:
        batch.close()


def test_queue_schedule_circular_boundary(mvd):
    """Circular boundary: the queue stages its tiles with plain L2 loads
    (indices wrapped) instead of TMA copies."""
    vols = synth.uneven_volumes(4, seed=310, side=(48, 130), planes=(2, 5), views=(2, 2), psf=(5, 35),
                                iters=(2, 4), density=2e-3, device="cuda")
    batch, ests = make_batch(mvd, vols, "sequential", boundary="circular")
    try:
        mvd.mvd_batch_set_schedule(batch, "queue")
        mvd.mvd_batch_run(batch)
        mvd.mvd_batch_device_status(batch)
        assert mvd.mvd_batch_queue_info(batch)["queue_volumes"] == 4
        check_against_oracle(vols, ests, "sequential", lambda P: [0, P - 1], boundary="circular")
    finally:
        batch.close()


def test_queue_schedule_full_plane_sizes(mvd):
    """Volumes 4, 12, 22, 27 and 46 of the 64-volume batch (seed 1000) at
    their full sizes (planes of 585, 595, 684, 511 and 109 px; 16 to 89
    planes; 2 to 4 views; PSFs 13 to 39 px; 10 to 20 iterations), views in
    sequence: the rank-1 volumes run on the queue (three size classes), the
    oblique ones as graph branches; two sampled planes per volume against
    the oracle."""
    vols = synth.uneven_volumes(64, seed=1000, only=[4, 12, 22, 27, 46], device="cuda")
    batch, ests = make_batch(mvd, vols, "sequential")
    try:
        mvd.mvd_batch_set_schedule(batch, "queue")
        mvd.mvd_batch_run(batch)
        mvd.mvd_batch_device_status(batch)
        info = mvd.mvd_batch_queue_info(batch)
        assert info["queue_volumes"] >= 3
        check_against_oracle(vols, ests, "sequential", lambda P: [1, P - 2])
    finally:
        batch.close()


def test_queue_wait_timeout_reaches_the_host(mvd):
    """A negative wait budget makes the first wait of every CTA report a
    timeout: the batch's status word reads MVD_ERR_TIMEOUT and the launch
    ends; with the default budget the same batch is correct again."""
    vols = synth.uneven_volumes(3, seed=320, side=(60, 90), planes=(2, 4), views=(2, 2), psf=(7, 15),
                                iters=(3, 4), density=2e-3, device="cuda")
    batch, ests = make_batch(mvd, vols, "sequential")
    try:
        mvd.mvd_batch_set_schedule(batch, "queue")
        mvd.mvd_batch_set_wait_budget(batch, -1)
        mvd.mvd_batch_run(batch)
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_batch_device_status(batch)
        assert ei.value.status == mvd.MVD_ERR_TIMEOUT
        mvd.mvd_batch_set_wait_budget(batch, 0)
        mvd.mvd_batch_run(batch)
        mvd.mvd_batch_device_status(batch)
        check_against_oracle(vols, ests, "sequential", lambda P: [0, P - 1])
    finally:
        batch.close()
