"""The benchmark line's `roofline.traffic` (DRAM bytes per launch from an ncu
capture) describes the kernels as they were captured: once a fused-kernel
source file differs from the captured state, the figure is reported as
null."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_reported_only_for_the_captured_sources(monkeypatch):
    recorded = bench.NCU_TRAFFIC_PER_LAUNCH["volume1024x4"]["blur_ratio"]
    monkeypatch.setattr(bench, "fused_sources_sha16", lambda: bench.NCU_TRAFFIC_SOURCE_SHA16)
    assert bench.ncu_traffic("volume1024x4", "blur_ratio") == recorded
    assert bench.ncu_traffic("volume512", "blur_ratio") is None      # no capture of that workload
    assert bench.ncu_traffic("volume1024x4", "reslice") is None        # no capture of that kernel
    monkeypatch.setattr(bench, "fused_sources_sha16", lambda: "0" * 16)
    assert bench.ncu_traffic("volume1024x4", "blur_ratio") is None


def test_source_hash_covers_every_listed_file():
    h = bench.fused_sources_sha16()
    assert len(h) == 16 and int(h, 16) >= 0
    for f in bench.FUSED_KERNEL_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_1503_07998_gb300", "csrc", f)), f
