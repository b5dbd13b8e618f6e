"""The paper's stream-count models (Sec. 2.2-2.4, Sec. 3) against the numbers
the paper prints in Tables 1, 2, 4 and 5."""
import math

import numpy as np

from oracle import heuristic as H


def test_table1_sum_is_eq3_and_gomez_luna_column(golden):
    for size, t1c, t1d, t3h, t3c, s, gl, actual in golden("table1_overlap_ops.txt"):
        total = H.overlap_sum(float(t1c), float(t1d), float(t3h), float(t3c))
        assert abs(total - float(s)) < 2e-6
        assert round(H.gomez_luna_streams(float(s)), 1) == float(gl)


def test_table2_eq5_overhead_and_slack(golden):
    best = None
    for S, tstr, tnon, s, tov, sl in golden("table2_streams_1e6.txt"):
        S, tstr, tnon, s, tov, sl = int(S), float(tstr), float(tnon), float(s), float(tov), float(sl)
        assert abs(H.t_overhead(tstr, tnon, S, s) - tov) < 2e-6
        assert abs(H.slack(S, s, tov) - sl) < 2e-6
        # the slack is also T_non_str - T_str
        assert abs((tnon - tstr) - sl) < 2e-6
        if best is None or sl > best[1]:
            best = (S, sl)
    assert best[0] == 8


def test_table2_rule_picks_the_highlighted_optimum(golden):
    table = {int(r[0]): float(r[4]) for r in golden("table2_streams_1e6.txt")}
    s = float(golden("table2_streams_1e6.txt")[0][3])
    assert H.optimum_streams(s, lambda S: table[S], candidates=(2, 4, 8, 16, 32)) == 8


def test_table4_every_prediction(golden):
    mismatches = []
    for size, n_act, n_pre in golden("table4_opt_streams.txt"):
        pred = H.predict_streams(float(size))
        assert pred == int(n_pre), (size, pred, n_pre)
        if int(n_act) != int(n_pre):
            mismatches.append(float(size))
    assert mismatches == [1e5, 5e5]  # the two the paper flags


def test_table4_hand_checked_slacks():
    # size 1e6 (small model): slack at S=8 beats S=16
    s = H.sum_model(1e6)
    sl8 = 7 / 8 * s - H.overhead_small(1e6, 8)
    sl16 = 15 / 16 * s - H.overhead_small(1e6, 16)
    assert sl8 > sl16 and abs(sl8 - 1.337) < 2e-3 and abs(sl16 - 1.302) < 2e-3
    # size 1e5: S=2 wins narrowly over S=1
    s = H.sum_model(1e5)
    assert abs((0.5 * s - H.overhead_small(1e5, 2)) - 0.040) < 1e-3
    assert abs((0.0 - H.overhead_small(1e5, 1)) - 0.038) < 1e-3


def test_big_model_reads_log2_of_s_to_the_four_thirds():
    for S in (2, 4, 8, 16, 32):
        lhs = H.overhead_big(2e7, S)
        k, q, r = H.OVERHEAD_BIG_2080TI
        assert math.isclose(lhs, (k * 2e7 + q) * math.log2(S ** (4 / 3)) + r, rel_tol=1e-12)


def test_eq2_reduces_to_eq1_with_one_stream_and_no_overhead():
    parts = (0.7, 1.1, 0.3, 2.2, 0.05, 0.9, 0.6)
    assert math.isclose(H.t_str(*parts, streams=1, t_overhead=0.0), H.t_non_str(*parts))
    # and the streamed part shrinks by S
    t4 = H.t_str(*parts, streams=4, t_overhead=0.0)
    s = H.overlap_sum(parts[1], parts[2], parts[4], parts[5])
    assert math.isclose(H.t_non_str(*parts) - t4, 0.75 * s)


def test_table5_fp32_half_rule(golden):
    n_half = n_same = 0
    for size, f32, f64, cmp in golden("table5_fp32_streams.txt"):
        f32, f64 = int(f32), int(f64)
        if cmp == "half":
            assert f32 == max(1, f64 // 2)
            n_half += 1
        else:
            assert f32 == f64
            n_same += 1
    assert (n_half, n_same) == (7, 10)
    assert H.predict_streams_fp32(1e6) == 4 and H.predict_streams_fp32(1e3) == 1


def test_refits_recover_known_coefficients():
    rng = np.random.default_rng(0)
    sizes = rng.uniform(1e3, 1e8, 50)
    k, q = H.fit_sum_model(sizes, [H.sum_model(s) for s in sizes])
    assert math.isclose(k, H.SUM_MODEL_2080TI[0], rel_tol=1e-9)
    assert math.isclose(q, H.SUM_MODEL_2080TI[1], rel_tol=1e-6)
    S = rng.choice([1, 2, 4, 8, 16, 32], 60).astype(float)
    sz = rng.uniform(1e3, 1e6, 60)
    fit = H.fit_overhead_small(sz, S, [H.overhead_small(a, b) for a, b in zip(sz, S)])
    np.testing.assert_allclose(fit, H.OVERHEAD_SMALL_2080TI, rtol=1e-8)
    sz = rng.uniform(2e6, 1e8, 60)
    fit = H.fit_overhead_big(sz, S, [H.overhead_big(a, b) for a, b in zip(sz, S)])
    np.testing.assert_allclose(fit, H.OVERHEAD_BIG_2080TI, rtol=1e-8)
    assert H.r_squared([1, 2, 3], [1, 2, 3]) == 1.0
