"""The paper's modelling pipeline (Sec. 2.4: Eq. 4 sum model, the two Eq. 7
overhead forms, the rule of Eq. 6, Table 6's metrics and Table 4's
predicted-vs-actual comparison) run on the committed GB300 host-pipeline
timings.  The package's fits and rule evaluation are pinned against the
oracle's independent fitting routines and rule, and the committed results
file against a recomputation."""
import json
import math
import os

import numpy as np
import pytest

from oracle import heuristic as H
from paper_2501_05938_gb300 import build as tps_build
from paper_2501_05938_gb300 import tune

PRED = os.path.join(os.path.dirname(tune.__file__), "predictor")


@pytest.fixture(scope="module")
def rows():
    tps_build.build()
    return tune.load(os.path.join(PRED, "timings_gb300.csv"))


@pytest.fixture(scope="module")
def res(rows):
    return tune.paper_models(rows)


def _train_points(rows, seed=tune.SPLIT_SEED, split=1e6):
    """The training subsets, rebuilt here from the raw samples."""
    smp = tune.paper_samples(rows)
    ns = sorted(smp)
    tr, _ = tune._split(len(ns), seed)
    sums = ([ns[i] for i in tr], [smp[ns[i]]["sum"] for i in tr])
    ov = {"small": [], "big": []}
    for n in ns:
        t1, sm = smp[n]["t"][1], smp[n]["sum"]
        for S, ts in sorted(smp[n]["t"].items()):
            if S > 1:
                ov["small" if n <= split else "big"].append((n, S, H.t_overhead(ts, t1, S, sm)))
    out = {}
    for name, pts in ov.items():
        tr2, _ = tune._split(len(pts), seed + (1 if name == "big" else 0))
        out[name] = [pts[i] for i in tr2]
    return sums, out


def test_fits_match_the_oracle_least_squares(rows, res):
    sums, ov = _train_points(rows)
    k, q = H.fit_sum_model(*sums)
    np.testing.assert_allclose(res["sum_model"]["coeffs"], [k, q], rtol=1e-9)
    sm = H.fit_overhead_small(*zip(*ov["small"]))
    np.testing.assert_allclose(res["overhead_small"]["coeffs"], sm, rtol=1e-9, atol=1e-15)
    bg = H.fit_overhead_big(*zip(*ov["big"]))
    np.testing.assert_allclose(res["overhead_big"]["coeffs"], bg, rtol=1e-9, atol=1e-15)


def test_metrics_match_the_oracle(rows, res):
    sums, ov = _train_points(rows)
    k, q = res["sum_model"]["coeffs"]
    pred = [k * n + q for n in sums[0]]
    assert res["sum_model"]["train"]["r2"] == pytest.approx(H.r_squared(sums[1], pred), abs=1e-12)
    co = res["overhead_small"]["coeffs"]
    y = [o for _, _, o in ov["small"]]
    yhat = [H.overhead_small(n, S, co) for n, S, _ in ov["small"]]
    m = res["overhead_small"]["train"]
    assert m["r2"] == pytest.approx(H.r_squared(y, yhat), abs=1e-12)
    mse = float(np.mean((np.array(y) - np.array(yhat)) ** 2))
    assert m["mse"] == pytest.approx(mse, rel=1e-9) and m["rmse"] == pytest.approx(math.sqrt(mse))


def test_rule_in_libtps_matches_the_oracle_rule(res):
    co = [res[k]["coeffs"] for k in ("sum_model", "overhead_small", "overhead_big")]
    for r in res["table"]:
        assert r["N_pre"] == H.predict_streams(r["n"], tuple(co[0]), tuple(co[1]), tuple(co[2]))
        assert r["N_pre_2080ti"] == H.predict_streams(r["n"])


def test_committed_results_are_reproduced(res):
    with open(os.path.join(PRED, "paper_models_gb300.json")) as f:
        saved = json.load(f)
    for k in ("sum_model", "overhead_small", "overhead_big"):
        np.testing.assert_allclose(saved[k]["coeffs"], res[k]["coeffs"], rtol=1e-12)
        for s in ("train", "test"):
            assert saved[k][s]["samples"] == res[k][s]["samples"]
            assert saved[k][s]["r2"] == pytest.approx(res[k][s]["r2"], abs=1e-12)
    assert [(r["n"], r["N_act"], r["N_pre"]) for r in saved["table"]] == \
        [(r["n"], r["N_act"], r["N_pre"]) for r in res["table"]]


def test_split_is_three_to_one_and_disjoint():
    tr, te = tune._split(23, 5)
    assert len(tr) == 18 and len(te) == 5
    assert sorted(np.concatenate([tr, te]).tolist()) == list(range(23))


def test_sum_model_is_near_perfect_as_in_the_paper(res):
    # Sec. 2.4: the overlapped sum is linear in the size (R-squared ~ 1)
    assert res["sum_model"]["test"]["r2"] > 0.999
    assert all(r["N_act"] in H.STREAM_CANDIDATES for r in res["table"])
