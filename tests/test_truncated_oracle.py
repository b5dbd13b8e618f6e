"""Pins of the truncated-decoupling oracle (oracle/truncated.py) to facts
independent of it: the untruncated case is the exact solution, windows
solved by dense elimination agree, the derived error bound holds on every
window of random dominant systems, and for a Toeplitz matrix the error
decays at the closed-form rate of its inverse."""
import math

import numpy as np
import pytest

import oracle
from oracle import truncated as T
from paper_2501_05938_gb300 import synth


def test_no_truncation_is_exact():
    s = synth.system(1, 5000)
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    for R, h in ((5000, 0), (100, 5000), (7, 6000)):
        x, bnd = T.truncated(s["a"], s["b"], s["c"], s["d"], R, h)
        np.testing.assert_array_equal(x, ref)
        assert np.all(bnd == 0.0)


def test_windows_match_dense_elimination():
    rng = np.random.default_rng(3)
    n, R, h = 37, 8, 3
    s = synth.system(2, n)
    x, _ = T.truncated(s["a"], s["b"], s["c"], s["d"], R, h)
    for k0, k1, e0, e1 in T.windows(n, R, h):
        m = e1 - e0
        A = np.zeros((m, m))
        for i in range(m):
            A[i, i] = s["b"][e0 + i]
            if i > 0:
                A[i, i - 1] = s["a"][e0 + i]
            if i < m - 1:
                A[i, i + 1] = s["c"][e0 + i]
        xw = np.linalg.solve(A, s["d"][e0:e1])
        np.testing.assert_allclose(x[k0:k1], xw[k0 - e0:k1 - e0], rtol=1e-13, atol=1e-14)
    assert rng is not None


@pytest.mark.parametrize("kind,ratio", [("paper", None), ("ratio", 1.1), ("ratio", 2.0)])
@pytest.mark.parametrize("h", [1, 2, 4, 8, 16])
def test_bound_holds_on_every_window(kind, ratio, h):
    n, R = 20000, 256
    if kind == "paper":
        s = synth.system(10 + h, n)
    else:
        s = synth.system(20 + h, n, kind=synth.KIND_RATIO, ratio=ratio)
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    x, bnd = T.truncated(s["a"], s["b"], s["c"], s["d"], R, h)
    xmax = np.max(np.abs(ref))
    for w, (k0, k1, _, _) in enumerate(T.windows(n, R, h)):
        err = np.max(np.abs(x[k0:k1] - ref[k0:k1]))
        assert err <= bnd[w] * xmax * (1 + 1e-9) + 1e-13 * xmax


def test_toeplitz_error_decays_at_the_inverse_rate():
    # a = c = 1, b = beta: the inverse decays like r^|i-j|, r = (beta - sqrt(beta^2 - 4)) / 2
    n, R, beta = 4000, 500, 3.0
    r = (beta - math.sqrt(beta * beta - 4.0)) / 2.0
    a = np.ones(n)
    c = np.ones(n)
    b = np.full(n, beta)
    rng = np.random.default_rng(7)
    xt = rng.uniform(-1, 1, n)
    d = b * xt
    d[1:] += a[1:] * xt[:-1]
    d[:-1] += c[:-1] * xt[1:]
    ref = oracle.thomas(a, b, c, d)
    errs = []
    for h in (8, 12):
        x, bnd = T.truncated(a, b, c, d, R, h)
        errs.append(np.max(np.abs(x - ref)))
        assert errs[-1] <= np.max(bnd) * np.max(np.abs(ref)) * (1 + 1e-9)
    rate = (errs[1] / errs[0]) ** (1.0 / 4.0)
    assert abs(rate - r) / r < 0.15, (rate, r)
    # the bound's rate q = 2 / beta is conservative: q >= r
    assert 2.0 / beta >= r
