"""Host-side logic of bench.py (no GPU): the roofline arithmetic of the JSON
line and the DRAM-traffic table, which is reported only while the kernel's
sources still hash to the captured version."""
import hashlib
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_roofline_hbm_kernel(monkeypatch):
    monkeypatch.setattr(bench, "measured_traffic", lambda k: None)
    steps, npts = 10, 200_000
    # per step: projection 0.2 ms in one launch, states 0.16 ms
    kern = {"bsc_proj_bf16": (2.0, 10), "bsc_states": (1.6, 10), "bsc_prep": (0.12, 10)}
    rl, shares = bench.roofline(kern, steps, 6792.7, "measured", npts)
    assert rl["kernel"] == "bsc_proj_bf16" and rl["bound"] == "hbm"
    expect = 4 * bench.D * npts / 0.2e-3 / 1e9          # Y read once, GB/s
    assert rl["achieved"] == pytest.approx(expect, rel=1e-12)
    assert rl["frac"] == pytest.approx(expect / 6792.7, rel=1e-12)
    assert rl["traffic"] is None
    assert sum(v["share"] for v in shares.values()) == pytest.approx(1.0)


def test_roofline_alu_kernel_per_launch(monkeypatch):
    monkeypatch.setattr(bench, "measured_traffic", lambda k: 1000.0)
    steps, npts = 4, 150_000
    # two launches per step: the per-launch time is what the work is divided by
    kern = {"bsc_proj_f32": (8.0, 8), "bsc_states": (1.0, 4)}
    rl, _ = bench.roofline(kern, steps, 6792.7, "measured", npts)
    assert rl["kernel"] == "bsc_proj_f32" and rl["bound"] == "alu"
    expect = bench.D * bench.H * npts / 1.0e-3 / 1e12
    assert rl["achieved"] == pytest.approx(expect, rel=1e-12)
    assert rl["frac"] == pytest.approx(expect / bench.ALU_PEAK_TOPS, rel=1e-12)
    assert rl["traffic"] == pytest.approx(1000.0 * npts)


def test_traffic_table_follows_the_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1908_06843_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("kernel v1\n")
    (csrc / "h.cuh").write_text("header\n")
    digest = hashlib.sha256(b"kernel v1\nheader\n").hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# comment\nbsc_states 139.2 k.cu,h.cuh " + digest + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("bsc_states") == pytest.approx(139.2)
    assert bench.measured_traffic("astat_tc") is None        # not in the table
    (csrc / "k.cu").write_text("kernel v2\n")                 # the kernel changed
    assert bench.measured_traffic("bsc_states") is None
