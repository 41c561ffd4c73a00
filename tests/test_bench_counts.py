"""The algorithmic operation counts bench.py divides by: the generic scheme counts only the
stages the result needs (Dormand-Prince 5's seventh stage has weight 0 and feeds nothing)."""
import numpy as np

import bench
import oracle


def test_rk4_counts():
    assert bench.FP64_INST_PER_SITE_STEP == 4 * 7 + 9 + 12
    assert bench.FP32K_INST_PER_SITE_STEP == 4 * 7 + 9 + 9 + 12


def test_generic_counts_skip_dead_stages():
    # Dormand-Prince 5, Roessler with second-neighbour coupling (10 operations per slope):
    # six needed stages with 1 + 2 + 3 + 4 + 5 stage-state terms, five nonzero weights
    assert bench.generic_fp_ops(bench.DOPRI5_A, bench.DOPRI5_B, 3, 10, False) == 15 * 3 + 6 * 10 + 5 * 3 + 3
    assert bench.generic_fp_ops(bench.DOPRI5_A, bench.DOPRI5_B, 3, 10, True) == 15 * 3 + 6 * 10 + 5 * 3 + 12
    # classical RK4 through the generic scheme: every stage needed
    assert bench.generic_fp_ops(oracle.RK4_A, oracle.RK4_B, 3, 7, False) == 3 * 3 + 4 * 7 + 4 * 3 + 3
    # a stage used only by a dead stage is dead too
    A = np.array([[0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]])
    b = np.array([1.0, 0, 0])
    assert bench.generic_fp_ops(A, b, 2, 5, False) == 0 * 2 + 1 * 5 + 1 * 2 + 2
