"""CPU checks of bench.py's helpers and of the paper's Table 2 as transcribed."""
import numpy as np


def test_fit_linear_recovers_intercept_and_slope():
    import bench
    B = np.array(bench.TABLE2_B, dtype=float)
    A, C = bench.fit_linear(B, 3e-6 + 2.5e-9 * B)
    assert abs(A - 3e-6) < 1e-15 and abs(C - 2.5e-9) < 1e-18


def test_paper_table2_matches_its_stated_gain():
    """Sec. 5 states that the gain tends to C_CPU / C_GPU = 17.2: the two slopes
    transcribed from Table 2 must reproduce it."""
    import bench
    t = bench.PAPER_TABLE2
    assert abs(t["cpu"]["C"] / t["gpu"]["C"] - t["gain_limit"]) < 0.05


def _golden_table2():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_table2.txt")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows[parts[0]] = [float(v) for v in parts[1:]]
    return rows


def test_golden_table2_is_self_consistent_and_matches_bench():
    """The Table 2 fixture reproduces the gain Sec. 5 states, and bench.py's
    copy of it (printed with the --table2 sweep) is the same."""
    import bench
    g = _golden_table2()
    gpu, cpu = g["gpu_cuda_fortran_gtx760"], g["cpu_i7_4770_3.4GHz"]
    assert abs(cpu[1] / gpu[1] - g["gain_limit"][0]) < 0.05
    t = bench.PAPER_TABLE2
    assert (t["gpu"]["A"], t["gpu"]["C"]) == tuple(gpu)
    assert (t["cpu"]["A"], t["cpu"]["C"]) == tuple(cpu)
