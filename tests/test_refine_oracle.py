"""Pins for the step-by-step mixed-precision refinement oracle."""
import pytest

import oracle
from oracle import refine
from paper_2501_05938_gb300 import synth


@pytest.mark.parametrize("ratio", [1.01, 1.1, 2.0])
def test_refinement_reaches_fp64_solution(ratio):
    s = synth.system(5005, 20000, kind=synth.KIND_RATIO, ratio=ratio)
    x, iters, ok = refine.refine(s["a"], s["b"], s["c"], s["d"])
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert ok
    assert oracle.rel_forward_error(x, ref) < 1e-12
    assert 1 <= iters <= 10


def test_weaker_dominance_needs_more_iterations():
    it = []
    for ratio in (2.0, 1.01):
        s = synth.system(5006, 20000, kind=synth.KIND_RATIO, ratio=ratio)
        it.append(refine.refine(s["a"], s["b"], s["c"], s["d"], tol=1e-15)[1])
    assert it[0] <= it[1]
