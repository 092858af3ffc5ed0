"""Host-side helpers of bench.py: the figures read from the particle kernel's ncu capture
are used only while the kernel sources match the capture, and the instruction-issue
roofline is the capture's per-particle count over the measured time against 4 warp
instructions per SM-cycle on 152 SMs."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_helpers_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_issue_roofline_arithmetic(bench, monkeypatch):
    monkeypatch.setattr(bench, "profiled_value", lambda key: 100.0 if key == "warp_instructions_per_particle" else None)
    r = bench.issue_roofline(2.0, 1e6, {"sm_mhz": 2000.0})
    # 1e8 warp instructions in 2 ms = 50 G/s against 152 x 4 x 2.0 G/s
    assert r["achieved"] == pytest.approx(50.0)
    assert r["peak"] == pytest.approx(1216.0)
    assert r["frac"] == pytest.approx(50.0 / 1216.0)
    assert bench.issue_roofline(2.0, 1e6, None)["sm_mhz"] == 2070.0


def test_profile_figures_follow_the_kernel_sources(bench, monkeypatch):
    assert bench.profiled_value("no_such_figure") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.profiled_value("dram_bytes_per_particle") is None
    assert bench.profiled_traffic(1000) is None
    assert bench.issue_roofline(1.0, 1000, None) is None
