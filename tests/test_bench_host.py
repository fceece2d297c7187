"""Host-side pieces of bench.py, on CPU: the closed-loop capacity estimate of
the serving leg and the FP64 flop model's bookkeeping."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_steady_throughput_leaves_out_ramp_and_tail():
    import bench
    # completions every 2 s of 100 cells from t = 5 s on; window 20 s; one late completion
    done = [(5.0 + 2.0 * k, 100) for k in range(8)] + [(30.0, 10_000)]
    lam, n = bench.steady_throughput(done, 20.0)
    assert n == 8
    # the 7 completions after the first, over 20 - 5 s
    assert lam == pytest.approx(700 / 15.0)


def test_steady_throughput_falls_back_for_short_windows():
    import bench
    lam, n = bench.steady_throughput([(12.0, 600), (9.0, 300)], 8.0)
    assert n == 0 and lam == pytest.approx(900 / 12.0)
    lam, n = bench.steady_throughput([(3.0, 300), (12.0, 600)], 8.0)
    assert n == 1 and lam == pytest.approx(900 / 12.0)
    assert bench.steady_throughput([], 8.0) == (0.0, 0)


def test_fp64_flop_model_adds_up_the_counters():
    """fp64_flops charges each counter its per-unit figure: one cell with one
    attempt, one right-hand side and nothing else costs the RHS plus the
    attempt's Nordsieck work; the FP32 form charges no LU and a refined solve."""
    import bench
    S, R, n = 12, 40, 13
    f_rhs = bench.RHS_FLOPS_FIXED + R * bench.RHS_FLOPS_PER_REACTION
    f_step = (3 * 4 / 2 + 2 * 4 + 3) * n + n
    st = np.zeros((8, 1), dtype=np.int32)
    st[0, 0] = 1          # one accepted step
    st[3, 0] = 1          # one right-hand side
    assert bench.fp64_flops(S, R, n, st, 64) == pytest.approx(f_rhs + f_step)
    st[5, 0] = 1          # one LU
    st[6, 0] = 1          # one Newton solve
    lu64 = (2 / 3) * n ** 3 + 0.5 * n * n
    assert bench.fp64_flops(S, R, n, st, 64) == pytest.approx(f_rhs + f_step + lu64 + 2 * n * n)
    assert bench.fp64_flops(S, R, n, st, 32) == pytest.approx(f_rhs + f_step + 2 * n * n + 5 * n)
