"""Batches of independent volumes of uneven size, view count, PSF size and
iteration count, run as one CUDA graph (mvd_batch_*): every volume equals
what a context of its own computes, and sampled planes match the oracle."""

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


def single(mvd, v, order):
    V, H, P, W = v["stacks"].shape
    ctx = mvd.mvd_create(V, v["psfs"], v["K"], H, W, v["iters"], "zero", 1e-6)
    try:
        mvd.mvd_set_update_order(ctx, order)
        planes = torch.empty((V, P, H, W), dtype=torch.uint16, device="cuda")
        mvd.mvd_reslice(ctx, v["stacks"], planes)
        est = torch.empty((P, H, W), device="cuda")
        mvd.mvd_deconvolve_planes(ctx, planes, est)
        torch.cuda.synchronize()
        return est.cpu().numpy(), planes
    finally:
        ctx.close()


@pytest.mark.parametrize("tune", [False, True])
def test_uneven_batch_matches_single_volumes_and_oracle(mvd, tune, tmp_path, monkeypatch):
    vols = synth.uneven_volumes(5, seed=70, side=(40, 120), planes=(3, 8), views=(2, 4), psf=(5, 15),
                                iters=(2, 5), density=2e-3, device="cuda")
    order = "sequential"
    ests = [torch.full((v["P"], v["H"], v["W"]), -1.0, device="cuda") for v in vols]
    batch = mvd.mvd_batch_create([{"stacks": v["stacks"], "psfs": v["psfs"], "iters": v["iters"], "estimate": e}
                                  for v, e in zip(vols, ests)], order=order)
    try:
        if tune:
            monkeypatch.setenv("MVD_TUNE_CACHE", str(tmp_path / "tune.txt"))
            mvd.mvd_batch_tune(batch)
        n0 = mvd.mvd_launch_count()
        mvd.mvd_batch_run(batch)
        mvd.mvd_batch_run(batch)          # replay of the captured graph
        torch.cuda.synchronize()
        info = mvd.mvd_batch_info(batch)
        assert info["graph_kernels"] > 0
        assert mvd.mvd_launch_count() - n0 == 2 * info["graph_kernels"]
        for v, e in zip(vols, ests):
            want, planes = single(mvd, v, order)
            if tune:
                # the tuner may pick another route than a context's default:
                # equal up to FP32 rounding
                assert_parity(e.cpu().numpy(), want, what="tuned batch vs single context")
            else:
                np.testing.assert_array_equal(e.cpu().numpy(), want)
            p = v["P"] // 2
            phi = planes[:, p].cpu().numpy()[:, None]
            ref = oracle.rl_planes(phi, v["psfs"], v["iters"], eps=1e-6, order=order)
            assert_parity(want[p][None], ref, what=f"volume {v['H']}x{v['P']} V={v['views']} K={v['K']}")
        if tune:
            assert (tmp_path / "tune.txt").read_text().strip() != ""
    finally:
        batch.close()
