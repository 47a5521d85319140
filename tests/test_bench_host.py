"""Host-side arithmetic of the benchmark's JSON line (no GPU)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_job_rate_counts_every_rank():
    # 2 ranks x 655,362 rays x 20 steps in 10 ms = 2621.448 Mrays/s
    assert abs(bench.job_rate(655362, 2, 20, 10.0) - 2621.448) < 1e-9


def test_alu_roofline_operation_count_and_peak():
    r = bench.alu_roofline(10.0, 2.0, 1e6, 1.0, 152, 2000.0)
    assert r["bound"] == "alu" and r["unit"] == "Tops/s"
    assert r["ops_per_ray"] == 20 * 4 * 10 + 40 * 2            # 880 operations per ray
    assert abs(r["achieved"] - 0.88) < 1e-12                   # 880e6 ops in 1 ms
    assert abs(r["peak"] - 152 * 128 * 2000e6 / 1e12) < 1e-12  # 38.912 Tops/s
    assert abs(r["frac"] - 0.88 / 38.912) < 1e-12
