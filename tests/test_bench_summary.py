"""The band launch's ncu summary as bench.py reads it: figures only for the
kernel source they were taken on, and the issue roofline's arithmetic."""
import hashlib
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BAND = os.path.join(ROOT, "paper_2411_12365_gb300", "csrc", "burr_band.cu")


def test_committed_summary_matches_the_band_source():
    s = bench.ncu_band_summary(BAND)
    assert s is not None, "profiles/k_band_1e9_r8_traffic.txt was taken on another band source"
    assert s["dram_bytes"] > 1e8 and s["warp_instructions"] > 1e9 and s["keys"] >= 1 << 20


def test_summary_of_another_source_is_ignored(tmp_path):
    p = tmp_path / "summary.txt"
    p.write_text("kernel_source_sha256_16: 0000000000000000\ndram_bytes_per_launch_captured: 5\n"
                 "n_keys_captured: 7\n")
    assert bench.ncu_band_summary(BAND, str(p)) is None
    h = hashlib.sha256(open(BAND, "rb").read()).hexdigest()[:16]
    p.write_text(f"kernel_source_sha256_16: {h}\ndram_bytes_per_launch_captured: 5\nn_keys_captured: 7\n")
    assert bench.ncu_band_summary(BAND, str(p)) == {"dram_bytes": 5.0, "warp_instructions": None, "keys": 7.0}


def test_issue_roofline_arithmetic():
    r = bench.issue_roofline(2.0e9, 4.0, 152, 2070.0)
    assert r["peak"] == pytest.approx(152 * 4 * 2.07e9)
    assert r["achieved"] == pytest.approx(5.0e11)
    assert r["frac"] == pytest.approx(5.0e11 / (152 * 4 * 2.07e9))
