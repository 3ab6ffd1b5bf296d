"""Host-side arithmetic of bench.py (no GPU): the HBM fractions of the field stages and the sort,
and the slicing of a particle read-back whose planes are packed by the count written."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_hbm_stage_summary():
    steps, cells, particles = 10, 128 ** 3, 3.0e7
    prof = {"b_half": [1.0, steps], "b_half2": [2.0, steps], "e_step": [3.0, steps], "zero_j": [0.5, steps],
            "push_deposit": [70.0, 2 * steps], "sort": [4.0, 3]}
    out = bench.hbm_stage_summary(prof, steps, cells, particles, 4)
    peak = out["peak_gbs"]
    assert peak > 0
    # b_half: 36 B per cell in 0.1 ms per step
    assert out["b_half"]["ms"] == 0.1
    assert out["b_half"]["algorithmic_bytes"] == 36 * cells
    assert abs(out["b_half"]["gbs"] - 36 * cells / 1e-4 / 1e9) < 0.1
    assert abs(out["e_step"]["frac"] - 60 * cells / 3e-4 / 1e9 / peak) < 1e-3
    # the sort moves 84 B per particle once every 4 steps
    assert abs(out["sort"]["algorithmic_bytes"] - 84 * particles / 4) < 1e-6
    assert abs(out["sort"]["gbs"] - 84 * particles / 4 / 4e-4 / 1e9) < 0.1
    assert "push_deposit" not in out
    # a stage that did not run is left out
    assert "b_half" not in bench.hbm_stage_summary({"b_half": [0.0, 0]}, steps, cells, particles, 1)


def test_planar_head_reads_planes_packed_by_count():
    cap, n = 7, 5
    buf = np.full((4, cap), -1.0)
    flat = buf.reshape(-1)
    want = np.arange(4 * n, dtype=float).reshape(4, n)
    flat[:4 * n] = want.reshape(-1)  # what the library writes: plane q at q * n
    got = bench.planar_head(buf, n)
    assert got.shape == (4, n) and np.array_equal(got, want)
    assert bench.planar_head(buf, 0).shape == (4, 0)
