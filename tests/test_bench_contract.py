"""The benchmark's roofline arithmetic, without a GPU: the algorithmic bytes
of one lattice update, the achieved bandwidth and fraction a line reports, and
the peak it divides by."""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_per_lattice_update():
    """Two components x 19 populations, each read once and written once: 304 B
    in float32; 16-bit storage keeps 18 moving offsets of 2 B and the float
    rest population per component: 160 B."""
    assert bench.ALG_BYTES_PER_LU == 2 * 19 * 2 * 4 == 304
    assert bench.ALG_BYTES_PER_LU_16 == 2 * (18 * 2 + 4) * 2 == 160


def test_roofline_fraction():
    nodes, ms, peak = 26_148_864, 1.978, 6770.1
    r = bench.roofline(304, nodes, ms, "passes", peak, "measured")
    assert r["algorithmic_bytes_per_launch"] == 304 * nodes
    assert r["achieved"] == pytest.approx(304 * nodes / (ms / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None


def test_peak_is_the_measured_copy_bandwidth():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        pytest.skip("no measured peaks in this checkout")
    peak, kind = bench.measured_peak()
    assert kind == "measured"
    assert peak == pytest.approx(float(json.load(open(path))["hbm_gbs"]))


def test_l2_note_names_the_working_set_against_l2():
    assert "exceeds" in bench.l2_note(7949e6)
    assert "does not exceed" in bench.l2_note(100e6)
