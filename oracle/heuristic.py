"""Stream-count time models and the optimum-stream rule -- TEST INFRASTRUCTURE.

Plain Python restatement of Sec. 2.2-2.4 of the paper (times in ms):

  Eq. 1  T_non_str = (T1_H2D + T1_COMP + T1_D2H) + T2_COMP + (T3_H2D + T3_COMP + T3_D2H)
  Eq. 2  T_str = T1_H2D + (T1_COMP + T1_D2H + T3_H2D + T3_COMP) / S
                 + T2_COMP + T3_D2H + T_overhead
  Eq. 3  sum = T1_COMP + T1_D2H + T3_H2D + T3_COMP
  Eq. 4  sum_model(size) = 2.1890017149e-6 * size + 0.1470644998564126
  Eq. 5  T_overhead = (T_str - T_non_str) + (S - 1) / S * sum
  Eq. 6  the optimum S satisfies T_overhead < (S - 1) / S * sum and has the
         largest slack (S - 1) / S * sum - T_overhead among those that do
  Eq. 7  T_overhead_small(size, S) = 2.245645331e-7 * size
                                    + 0.6009426920043296 * log10(S) - 0.0605183610625299
         T_overhead_big(size, S)   = (3.56594859e-8 * size + 0.0522781620855163)
                                    * log2(S ** (4/3)) + 0.3941472844770443
         (small for size <= 1e6, big for size > 1e6)
  Sec. 2.3  Gomez-Luna et al.: T_overhead = S * tau, optimum S* = sqrt(sum / tau),
            tau = 0.004448 ms on the RTX 2080 Ti.
  Sec. 2.1  only S in {1, 2, 4, 8, 16, 32} (32 hardware queues).
  Sec. 3.2  for FP32 the recommendation is half the FP64 optimum.

Readings (the paper leaves these implicit):
  * the candidate set of Eq. 6 includes S = 1, whose slack is -T_overhead(1);
    when no candidate satisfies the inequality the answer is S = 1;
  * log2(S^(4/3)) is (4/3) * log2(S);
  * halving never goes below one stream.
"""
from __future__ import annotations

import math

STREAM_CANDIDATES = (1, 2, 4, 8, 16, 32)
TAU_2080TI_MS = 0.004448

SUM_MODEL_2080TI = (2.1890017149e-6, 0.1470644998564126)
OVERHEAD_SMALL_2080TI = (2.245645331e-7, 0.6009426920043296, -0.0605183610625299)
OVERHEAD_BIG_2080TI = (3.56594859e-8, 0.0522781620855163, 0.3941472844770443)
SMALL_BIG_SPLIT = 1e6


def t_non_str(t1_h2d, t1_comp, t1_d2h, t2_comp, t3_h2d, t3_comp, t3_d2h):
    """Eq. 1."""
    return (t1_h2d + t1_comp + t1_d2h) + t2_comp + (t3_h2d + t3_comp + t3_d2h)


def t_str(t1_h2d, t1_comp, t1_d2h, t2_comp, t3_h2d, t3_comp, t3_d2h, streams, t_overhead):
    """Eq. 2 (a lower bound; exact for big sizes)."""
    return (t1_h2d + (t1_comp + t1_d2h + t3_h2d + t3_comp) / streams + t2_comp + t3_d2h
            + t_overhead)


def overlap_sum(t1_comp, t1_d2h, t3_h2d, t3_comp):
    """Eq. 3."""
    return t1_comp + t1_d2h + t3_h2d + t3_comp


def sum_model(size, coeffs=SUM_MODEL_2080TI):
    """Eq. 4 (linear regression of the overlapped sum on the SLAE size)."""
    k, q = coeffs
    return k * size + q


def t_overhead(t_str_ms, t_non_str_ms, streams, sum_ms):
    """Eq. 5."""
    return (t_str_ms - t_non_str_ms) + (streams - 1) / streams * sum_ms


def slack(streams, sum_ms, t_overhead_ms):
    """Right-hand side of Eq. 6 minus T_overhead."""
    return (streams - 1) / streams * sum_ms - t_overhead_ms


def overhead_small(size, streams, coeffs=OVERHEAD_SMALL_2080TI):
    """Eq. 7, model for sizes <= 1e6."""
    k, q, r = coeffs
    return k * size + q * math.log10(streams) + r


def overhead_big(size, streams, coeffs=OVERHEAD_BIG_2080TI):
    """Eq. 7, model for sizes > 1e6; log2(S^(4/3)) read as (4/3) log2 S."""
    k, q, r = coeffs
    return (k * size + q) * (4.0 / 3.0) * math.log2(streams) + r


def overhead_model(size, streams, small=OVERHEAD_SMALL_2080TI, big=OVERHEAD_BIG_2080TI,
                   split=SMALL_BIG_SPLIT):
    return overhead_small(size, streams, small) if size <= split else overhead_big(size, streams, big)


def optimum_streams(sum_ms, overhead_of_s, candidates=STREAM_CANDIDATES):
    """Eq. 6: among S with T_overhead(S) < (S-1)/S * sum pick the largest slack.

    ``overhead_of_s`` maps S -> T_overhead(S).  Returns 1 when no candidate
    satisfies the inequality.
    """
    best_s, best_slack = None, None
    for s in candidates:
        ov = overhead_of_s(s)
        rhs = (s - 1) / s * sum_ms
        if ov < rhs:
            sl = rhs - ov
            if best_slack is None or sl > best_slack:
                best_s, best_slack = s, sl
    return 1 if best_s is None else best_s


def predict_streams(size, sum_coeffs=SUM_MODEL_2080TI, small=OVERHEAD_SMALL_2080TI,
                    big=OVERHEAD_BIG_2080TI, split=SMALL_BIG_SPLIT,
                    candidates=STREAM_CANDIDATES):
    """The paper's heuristic: Eq. 4 and Eq. 7 fed into the rule of Eq. 6."""
    s_model = sum_model(size, sum_coeffs)
    return optimum_streams(s_model, lambda s: overhead_model(size, s, small, big, split),
                           candidates)


def predict_streams_fp32(size, **kw):
    """Sec. 3.2: half the FP64 optimum, at least one stream."""
    return max(1, predict_streams(size, **kw) // 2)


def gomez_luna_streams(sum_ms, tau_ms=TAU_2080TI_MS):
    """Sec. 2.3: S* = sqrt(sum / tau) from T_overhead = S * tau."""
    return math.sqrt(sum_ms / tau_ms)


# ---------------------------------------------------------------------------
# Refitting the models on new timings (Sec. 2.4 does this with scikit-learn's
# linear regression and SciPy's curve_fit on preset forms).
# ---------------------------------------------------------------------------

def fit_sum_model(sizes, sums):
    """Least-squares line sum = k * size + q (the form of Eq. 4)."""
    import numpy as np

    x = np.asarray(sizes, dtype=np.float64)
    y = np.asarray(sums, dtype=np.float64)
    A = np.stack([x, np.ones_like(x)], axis=1)
    (k, q), *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(k), float(q)


def fit_overhead_small(sizes, streams, overheads):
    """Least squares on the form of Eq. 7 (small): k*size + q*log10(S) + r."""
    import numpy as np

    x = np.asarray(sizes, dtype=np.float64)
    s = np.asarray(streams, dtype=np.float64)
    y = np.asarray(overheads, dtype=np.float64)
    A = np.stack([x, np.log10(s), np.ones_like(x)], axis=1)
    (k, q, r), *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(k), float(q), float(r)


def fit_overhead_big(sizes, streams, overheads):
    """Least squares on the form of Eq. 7 (big): (k*size + q)*(4/3)log2(S) + r."""
    import numpy as np

    x = np.asarray(sizes, dtype=np.float64)
    s = np.asarray(streams, dtype=np.float64)
    y = np.asarray(overheads, dtype=np.float64)
    g = (4.0 / 3.0) * np.log2(s)
    A = np.stack([x * g, g, np.ones_like(x)], axis=1)
    (k, q, r), *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(k), float(q), float(r)


def r_squared(y_true, y_pred):
    import numpy as np

    y_true = np.asarray(y_true, dtype=np.float64)
    y_pred = np.asarray(y_pred, dtype=np.float64)
    ss_res = float(np.sum((y_true - y_pred) ** 2))
    ss_tot = float(np.sum((y_true - np.mean(y_true)) ** 2))
    return 1.0 - ss_res / ss_tot if ss_tot > 0 else 0.0
