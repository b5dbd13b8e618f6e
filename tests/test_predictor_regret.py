"""What the trained predictor gains: regret against exhaustive search on the
held-out points of the GB300 timing sweep (odd exponents, 3 * 2^k sizes, an
unseen batch count), recomputed on the host from the committed timings and
weights through libtps's own inference, compared with the paper's stream
rule refit on the same timings and with the fixed defaults."""
import os

import pytest

from paper_2501_05938_gb300 import build as tps_build
from paper_2501_05938_gb300 import tune

PRED = os.path.join(os.path.dirname(tune.__file__), "predictor")


@pytest.fixture(scope="module")
def result():
    tps_build.build()
    rows = tune.load(os.path.join(PRED, "timings_gb300.csv"))
    return tune.evaluate(rows, os.path.join(PRED, "weights.bin"))


def test_predictor_regret_within_five_percent(result):
    summary, detail, _ = result
    assert summary["mlp"]["points"] >= 40
    assert summary["mlp"]["mean"] <= 0.05


def test_predictor_beats_the_method_without_it(result):
    summary, _, _ = result
    assert summary["mlp"]["mean"] < summary["defaults"]["mean"]
    assert summary["mlp"]["mean"] < summary["paper_rule"]["mean"]


def test_held_out_points_cover_every_kind(result):
    _, detail, _ = result
    kinds = {(d["kind"], d["dtype"]) for d in detail}
    assert {("device", 0), ("device", 1), ("host", 0), ("host", 1), ("batched", 0)} <= kinds
