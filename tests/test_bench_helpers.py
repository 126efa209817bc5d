"""Host-side arithmetic of bench.py's roofline records (no GPU work)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def test_plane_pass_bytes_135_three_loads():
    # 135^3, 3 loads, FP32: r, p, x vectors 3 x 3 x 135^3 x 4 B each; the half
    # spectrum 3 x 3 x 135 x 135 x 68 complex FP32 entries; one phase byte per voxel
    M = 135 ** 3
    vec = 3 * 3 * M * 4
    spec = 3 * 3 * 135 * 135 * 68 * 8
    fwd, strided, inv = bench.plane_pass_bytes((135, 135, 135), 3, 4)
    assert fwd == 2 * vec + M + spec
    assert strided == 2 * spec
    assert inv == spec + 6 * vec
    assert (fwd, strided, inv) == (268836975, 178459200, 620670600)


def test_per_pass_roofline():
    rows = bench.per_pass_roofline(["a", "b", "c"], [2e9, 1e9, 5e8], [1.0, 0.0, 0.5], 4000.0)
    assert [r["pass"] for r in rows] == ["a", "b", "c"]
    assert rows[0]["achieved_gbs"] == pytest.approx(2000.0)
    assert rows[0]["frac"] == pytest.approx(0.5)
    assert rows[1]["achieved_gbs"] is None and rows[1]["frac"] is None
    assert rows[2]["frac"] == pytest.approx(0.25)
    assert rows[2]["bytes"] == 500000000
