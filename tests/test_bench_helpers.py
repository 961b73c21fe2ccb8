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
