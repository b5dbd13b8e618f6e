"""Pins for the CPU oracle: each check comes from outside the oracle itself
(a LAPACK routine, a closed form, brute force, or an invariant of the
mathematics), so that a dropped term, a wrong sign, a shifted index or a
transposed operand in the oracle fails at least one of them."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2501_05938_gb300 import synth


def sdd(n, seed, kind=synth.KIND_PAPER, ratio=2.0):
    s = synth.system(seed, n, kind=kind, ratio=ratio)
    return s["a"], s["b"], s["c"], s["d"], s["x_true"]


def lapack_banded(a, b, c, d):
    """LAPACK gbsv through scipy: an independent tridiagonal solve."""
    n = b.shape[0]
    ab = np.zeros((3, n))
    ab[0, 1:] = c[:-1]
    ab[1, :] = b
    ab[2, :-1] = a[1:]
    return scipy.linalg.solve_banded((1, 1), ab, d)


def dense(a, b, c):
    n = b.shape[0]
    A = np.diag(b)
    if n > 1:
        A += np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    return A


# ---------------------------------------------------------------- closed forms
def test_thomas_n1_is_d_over_b():
    x = oracle.thomas([0.0], [4.0], [0.0], [3.0])
    assert x[0] == 0.75


def test_thomas_2x2_cramer():
    # [[b0, c0], [a1, b1]] x = d  ->  Cramer's rule
    a = np.array([0.0, 0.3]); b = np.array([2.0, -1.7]); c = np.array([0.5, 0.0])
    d = np.array([1.1, 0.4])
    det = b[0] * b[1] - c[0] * a[1]
    ref = np.array([(d[0] * b[1] - c[0] * d[1]) / det, (b[0] * d[1] - a[1] * d[0]) / det])
    for fn in (oracle.thomas, oracle.dense_ge, lambda *v: oracle.partition(*v, m=2),
               lambda *v: oracle.partition(*v, m=5)):
        np.testing.assert_allclose(fn(a, b, c, d), ref, rtol=1e-15, atol=0)


def test_3x3_cramer():
    a = np.array([0.0, 1.0, -2.0]); b = np.array([4.0, 5.0, 6.0]); c = np.array([1.0, 2.0, 0.0])
    d = np.array([1.0, 2.0, 3.0])
    A = dense(a, b, c)
    det = np.linalg.det(A)
    ref = []
    for j in range(3):
        Aj = A.copy(); Aj[:, j] = d
        ref.append(np.linalg.det(Aj) / det)
    # the determinant expansion by hand: 4*(5*6 - 2*(-2)) - 1*(1*6 - 0) = 130
    assert abs(det - 130.0) < 1e-12
    for fn in (oracle.thomas, oracle.dense_ge) + tuple(
            (lambda *v, m=m: oracle.partition(*v, m=m)) for m in (2, 3, 4)):
        np.testing.assert_allclose(fn(a, b, c, d), ref, rtol=1e-14, atol=1e-15)


def test_residual_by_hand():
    a = np.array([0.0, 1.0, 2.0]); b = np.array([3.0, 4.0, 5.0]); c = np.array([6.0, 7.0, 0.0])
    d = np.array([10.0, 20.0, 30.0]); x = np.array([1.0, 2.0, 3.0])
    # A x = [3+12, 1+8+21, 4+15] = [15, 30, 19]
    np.testing.assert_array_equal(oracle.residual(a, b, c, d, x), [-5.0, -10.0, 11.0])


def test_rel_forward_error_by_hand():
    assert oracle.rel_forward_error(np.array([1.0, 2.5]), np.array([1.0, 2.0])) == 0.25
    assert oracle.rel_forward_error(np.array([np.nan, 2.0]), np.array([1.0, 2.0])) == np.inf


# ------------------------------------------------ library routine (LAPACK gbsv)
@pytest.mark.parametrize("n", [1, 2, 3, 17, 256, 4099])
def test_thomas_matches_lapack(n):
    a, b, c, d, _ = sdd(n, 7 + n)
    ref = lapack_banded(a, b, c, d)
    assert oracle.rel_forward_error(oracle.thomas(a, b, c, d), ref) < 1e-14


@pytest.mark.parametrize("n,m", [(1000, 10), (4099, 32), (65536, 256), (777, 776), (50, 1000)])
def test_partition_matches_lapack(n, m):
    a, b, c, d, _ = sdd(n, 100 + n)
    ref = lapack_banded(a, b, c, d)
    assert oracle.rel_forward_error(oracle.partition(a, b, c, d, m), ref) < 1e-14


def test_dense_ge_matches_numpy_solve():
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 33, 64):
        a, b, c, d, _ = sdd(n, 200 + n)
        ref = np.linalg.solve(dense(a, b, c), d)
        assert oracle.rel_forward_error(oracle.dense_ge(a, b, c, d), ref) < 1e-14
    # a matrix that needs row interchanges: zero leading pivot
    a = np.array([0.0, 1.0, 1.0]); b = np.array([0.0, 1.0, 3.0]); c = np.array([1.0, 2.0, 0.0])
    d = rng.uniform(-1, 1, 3)
    ref = np.linalg.solve(dense(a, b, c), d)
    np.testing.assert_allclose(oracle.dense_ge(a, b, c, d), ref, rtol=1e-14)
    with pytest.raises(oracle.OracleError):
        oracle.thomas(a, b, c, d)


# ------------------------------------------------ brute force over m and L
def test_partition_every_block_size_and_tail_against_dense_ge():
    """Every n <= 40 and every m in 2..n+2 (so every last-block length L in
    1..m appears), against dense Gaussian elimination with pivoting."""
    for n in range(1, 41):
        a, b, c, d, _ = sdd(n, 300 + n)
        ref = oracle.dense_ge(a, b, c, d)
        for m in range(2, n + 3):
            x = oracle.partition(a, b, c, d, m)
            err = oracle.rel_forward_error(x, ref)
            assert err < 5e-15, (n, m, err)


def test_partition_64_slices_against_dense_ge():
    """The paper-shaped system (n = 65536, m = 256) cut into 64-row slices:
    each slice is its own tridiagonal system, solved by partition (m = 8, 13)
    and by dense elimination."""
    s = synth.system(1001, 65536)
    for start in range(0, 65536, 4096):
        sl = slice(start, start + 64)
        a, b, c, d = (s[k][sl].copy() for k in "abcd")
        a[0] = 0.0; c[-1] = 0.0
        ref = oracle.dense_ge(a, b, c, d)
        for m in (8, 13):
            assert oracle.rel_forward_error(oracle.partition(a, b, c, d, m), ref) < 5e-15


# ------------------------------------------------ manufactured solution / residual
@pytest.mark.parametrize("n,m", [(65536, 256), (100003, 32), (4096, 1024)])
def test_manufactured_solution_and_residual(n, m):
    a, b, c, d, xt = sdd(n, 1001 + n)
    # kappa_inf(A) <= ||A|| ||A^-1|| <= 6 * 1 for this generator (dominance >= 1)
    for x in (oracle.thomas(a, b, c, d), oracle.partition(a, b, c, d, m)):
        assert oracle.rel_forward_error(x, xt) < 6 * 64 * np.finfo(float).eps
        assert oracle.rel_residual(a, b, c, d, x) < 8 * np.finfo(float).eps
        assert oracle.normwise_backward_error(a, b, c, d, x) < 4 * np.finfo(float).eps


def test_partition_with_m_at_least_n_is_thomas():
    a, b, c, d, _ = sdd(500, 5)
    x1 = oracle.partition(a, b, c, d, 500)
    x2 = oracle.partition(a, b, c, d, 10**6)
    xt = oracle.thomas(a, b, c, d)
    assert oracle.rel_forward_error(x1, xt) < 1e-15
    assert oracle.rel_forward_error(x2, xt) < 1e-15


def test_ill_conditioned_ratio_generator():
    a, b, c, d, xt = sdd(20000, 9, kind=synth.KIND_RATIO, ratio=1.01)
    ref = lapack_banded(a, b, c, d)
    for x in (oracle.thomas(a, b, c, d), oracle.partition(a, b, c, d, 64)):
        assert oracle.rel_forward_error(x, ref) < 1e-12
        assert oracle.rel_residual(a, b, c, d, x) < 1e-14


# ------------------------------------------------ the reduced system
@pytest.mark.parametrize("n,m", [(1000, 10), (1001, 10), (1002, 10), (64, 64), (5000, 7)])
def test_reduced_system_is_sdd_and_holds_the_interface_values(n, m):
    a, b, c, d, _ = sdd(n, 40 + n)
    x_full = lapack_banded(a, b, c, d)
    x, (ra, rb, rc, rd) = oracle.partition(a, b, c, d, m, return_reduced=True)
    p = -(-n // m)
    assert ra.shape[0] == oracle.reduced_size(n, m) == 2 * p - (1 if n - (p - 1) * m == 1 else 0)
    # strictly diagonally dominant (a Schur complement of an SDD matrix)
    assert np.all(np.abs(rb) > np.abs(ra) + np.abs(rc))
    assert ra[0] == 0.0 and rc[-1] == 0.0
    # interface unknowns in the order f_0, l_0, f_1, l_1, ...
    idx = []
    for k in range(p):
        r0, r1 = k * m, min(k * m + m, n) - 1
        idx.append(r0)
        if r1 > r0:
            idx.append(r1)
    xr = lapack_banded(ra, rb, rc, rd)
    assert oracle.rel_forward_error(xr, x_full[idx]) < 1e-14
    # and the reduced rows hold for the exact interface values
    r = oracle.residual(ra, rb, rc, rd, x_full[idx])
    assert np.max(np.abs(r)) < 1e-13


# ------------------------------------------------ the pins are sensitive
def test_pins_catch_planted_mistakes():
    """Plausible mistakes (transposed a/c, flipped sign, shifted index) give
    solutions that the residual and LAPACK checks above reject."""
    a, b, c, d, _ = sdd(300, 77)
    ref = lapack_banded(a, b, c, d)
    wrong = [
        oracle.thomas(np.r_[0.0, c[:-1]], b, np.r_[a[1:], 0.0], d),  # sub/super swapped
        oracle.thomas(-a, b, c, d),                                   # sign of a
        oracle.thomas(np.r_[0.0, 0.0, a[1:-1]], b, c, d),             # a shifted by a row
    ]
    for x in wrong:
        assert oracle.rel_forward_error(x, ref) > 1e-3
        assert oracle.rel_residual(a, b, c, d, x) > 1e-3


def test_batched_thomas_decouples_systems():
    sizes = np.array([1, 2, 5, 300, 17, 1])
    off = synth.offsets_from_sizes(sizes)
    s = synth.system(11, int(off[-1]), offsets=off)
    x = oracle.thomas_batched(off, s["a"], s["b"], s["c"], s["d"])
    for i in range(len(sizes)):
        lo, hi = off[i], off[i + 1]
        ref = lapack_banded(s["a"][lo:hi], s["b"][lo:hi], s["c"][lo:hi], s["d"][lo:hi])
        assert oracle.rel_forward_error(x[lo:hi], ref) < 1e-14
    assert oracle.rel_forward_error(x, s["x_true"]) < 1e-13


def test_thomas_f32_is_single_precision():
    a, b, c, d, _ = sdd(5000, 3)
    x64 = oracle.thomas(a, b, c, d)
    x32 = oracle.thomas_f32(a, b, c, d)
    assert x32.dtype == np.float32
    err = oracle.rel_forward_error(x32.astype(np.float64), x64)
    assert 1e-9 < err < 6 * 64 * np.finfo(np.float32).eps


@pytest.mark.parametrize("n,m,threads", [(1000, 7, 3), (100003, 128, 8), (65, 64, 4),
                                         (2, 2, 16), (1, 5, 2), (4097, 32, 1)])
def test_threaded_partition_is_the_serial_partition(n, m, threads):
    """The multi-core CPU baseline runs the serial oracle's per-block
    arithmetic in the same order, so its x is the same bits (and is pinned
    through the serial partition's own pins)."""
    s = synth.system(90 + n, n)
    x1 = oracle.partition(s["a"], s["b"], s["c"], s["d"], m)
    x2 = oracle.partition_threaded(s["a"], s["b"], s["c"], s["d"], m, threads=threads)
    np.testing.assert_array_equal(x2, x1)
