"""Range of the double-float arithmetic (TPS_F64_DF) through the C ABI.

A double-float value is a pair of binary32 numbers, so it keeps full
precision only over about [2^-103, 2^127].  The solver scales every fp64
row exactly by the power of two that brings its diagonal entry into [1, 2),
and d (hence x) by a further 2^26; what is left is checked and reported as
TPS_ERR_RANGE: an entry above 2^84 |b| or not finite, a system whose |d / b|
is below 2^-84 in every row, an entry taken as 0 in a row that dominates
the system, an x at or above 2^101.  These tests scale the paper's systems
by powers of two -- whole rows (x unchanged, at any magnitude fp64 holds),
the right-hand side alone (x scaled), single rows -- and require either a
result that matches the fp64 Thomas oracle (relative forward error <= 1e-10,
relative residual <= 1e-12) or the range status, never TPS_OK with a wrong
x.  Every route is covered: the level-by-level solve, the single-launch
on-chip solve, the one-warp solve, packed batches, the host pipeline, the
windowed approximation and the allocation-free entry point.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2501_05938_gb300 import binding, synth

pytestmark = pytest.mark.gpu

FWD, RES = 1e-10, 1e-12
ROUTES = {"levels": binding.NO_ONCHIP, "onchip": 0}


def dev(v):
    return torch.as_tensor(np.ascontiguousarray(v)).to(device="cuda", dtype=torch.float64)


def solve(s, dtype="f64_df", flags=0, m=64):
    n = len(s["b"])
    a, b, c, d = (dev(s[k]) for k in "abcd")
    x = torch.full_like(b, float("nan"))
    plan = binding.Plan(n, dtype=dtype, m=m, flags=flags)
    plan.solve(a, b, c, d, x)
    torch.cuda.synchronize()
    return x.cpu().numpy(), plan.query()


def assert_matches(s, x):
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x, ref) <= FWD
    assert oracle.rel_residual(s["a"], s["b"], s["c"], s["d"], x) <= RES


def scaled(s, rows=1.0, rhs=1.0):
    """rows: a factor (or per-row factors) on a, b, c, d; rhs: on d alone."""
    t = dict(s)
    for k in "abc":
        t[k] = s[k] * rows
    t["d"] = s["d"] * rows * rhs
    return t


@pytest.mark.parametrize("route", ROUTES)
@pytest.mark.parametrize("n", [1000, 100003, 1 << 20])
@pytest.mark.parametrize("e", [-900, -500, -130, -100, 100, 130, 500, 900])
def test_row_scaling_leaves_x_bit_identical(route, n, e):
    """Whole rows times 2^e: the solve normalises each row by its diagonal's
    exponent, so every intermediate -- and x -- is the same bits."""
    s = synth.system(7000 + n, n)
    x0, info0 = solve(s, flags=ROUTES[route])
    x1, info1 = solve(scaled(s, rows=2.0 ** e), flags=ROUTES[route])
    assert info0["status"] == 0 and info1["status"] == 0, info1
    np.testing.assert_array_equal(x1, x0)
    assert_matches(s, x1)


@pytest.mark.parametrize("route", ROUTES)
def test_per_row_scales_leave_x_bit_identical(route):
    n = 262147
    s = synth.system(71, n)
    k = np.random.default_rng(71).integers(-900, 900, n)
    x0, _ = solve(s, flags=ROUTES[route])
    x1, info = solve(scaled(s, rows=np.ldexp(1.0, k)), flags=ROUTES[route])
    assert info["status"] == 0
    np.testing.assert_array_equal(x1, x0)


@pytest.mark.parametrize("route", ROUTES)
@pytest.mark.parametrize("e", [-80, -60, 60, 80])
def test_rhs_scaling_inside_the_range_matches(route, e):
    """d times 2^e scales x by 2^e; with max |d / b| inside [2^-84, 2^84]
    the pairs keep their precision, so the result meets the fp64 bar."""
    n = 100003
    s = scaled(synth.system(72, n), rhs=2.0 ** e)
    x, info = solve(s, flags=ROUTES[route])
    assert info["status"] == 0, info
    assert_matches(s, x)


@pytest.mark.parametrize("route", ROUTES)
@pytest.mark.parametrize("e", [-130, -100, -90, 90, 100, 130])
def test_rhs_scaling_outside_the_range_is_reported(route, e):
    """|d / b| below 2^-84 everywhere, or above 2^84 somewhere: the range
    status (and never TPS_OK with a wrong x); the plain fp64 solve serves it."""
    n = 100003
    s = scaled(synth.system(73, n), rhs=2.0 ** e)
    x, info = solve(s, flags=ROUTES[route])
    assert info["status_name"] == "TPS_ERR_RANGE", info
    x, info = solve(s, dtype="f64", flags=ROUTES[route])
    assert info["status"] == 0
    assert_matches(s, x)


@pytest.mark.parametrize("route", ROUTES)
def test_range_report_is_per_solve(route):
    """An out-of-range solve leaves nothing behind: the next solve on the
    same plan, in range, reports TPS_OK and matches."""
    n = 5000
    good = synth.system(74, n)
    bad = scaled(good, rhs=2.0 ** -120)
    plan = binding.Plan(n, dtype="f64_df", m=32, flags=ROUTES[route])
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    for s, want in ((bad, "TPS_ERR_RANGE"), (good, "TPS_OK"), (bad, "TPS_ERR_RANGE"),
                    (good, "TPS_OK")):
        plan.solve(*(dev(s[k]) for k in "abcd"), x)
        assert plan.query()["status_name"] == want
    assert_matches(good, x.cpu().numpy())


@pytest.mark.parametrize("route", ROUTES)
def test_small_and_zero_entries_are_not_flagged(route):
    """Entries of a, c, d far below their row's diagonal (taken as 0 by the
    pairs) or zero lose nothing that matters in the infinity norm when the
    row is of the system's scale: no range status, and the result matches."""
    n = 100003
    s = synth.system(75, n)
    rng = np.random.default_rng(75)
    idx = rng.choice(n, 4000, replace=False)
    s["d"][idx[:1000]] *= 2.0 ** -300  # taken as 0: far below the system's scale
    s["d"][idx[1000:2000]] = 0.0
    s["a"][idx[2000:3000]] *= 2.0 ** -200
    s["c"][idx[3000:]] *= 2.0 ** -120
    x, info = solve(s, flags=ROUTES[route])
    assert info["status"] == 0, info
    assert_matches(s, x)
    z = dict(s, d=np.zeros(n))  # d = 0 everywhere: x = 0 exactly
    x, info = solve(z, flags=ROUTES[route])
    assert info["status"] == 0 and not np.any(x), info


@pytest.mark.parametrize("route", ROUTES)
@pytest.mark.parametrize("where", ["a", "c", "d"])
@pytest.mark.parametrize("bad", [np.inf, np.nan, 2.0 ** 90])
def test_entry_out_of_range_is_reported(route, where, bad):
    n = 100003
    s = synth.system(76, n)
    s[where][n // 3] = bad
    _, info = solve(s, flags=ROUTES[route])
    assert info["status_name"] == "TPS_ERR_RANGE", info


@pytest.mark.parametrize("route", ROUTES)
@pytest.mark.parametrize("dtype", ["f64", "f64_df"])
def test_unused_entries_are_not_checked(route, dtype):
    """a[0] and c[n-1] are never read: non-finite values there change nothing."""
    n = 100003
    s = synth.system(77, n)
    x0, _ = solve(s, dtype=dtype, flags=ROUTES[route])
    s["a"][0], s["c"][n - 1] = np.nan, np.inf
    x1, info = solve(s, dtype=dtype, flags=ROUTES[route])
    assert info["status"] == 0, info
    np.testing.assert_array_equal(x1, x0)


@pytest.mark.parametrize("route", ROUTES)
def test_dominant_row_is_reported_or_served(route):
    """b = 1e300 in one row with a, c, d of order 1: scaled by its diagonal
    the row's other entries fall below the pairs' range, and with them x of
    that row (about 1e-300); x is still right to 1e-300 in the infinity
    norm, but b x of that row is of order 1, so the residual bar cannot be
    met and the range is reported.  The whole row scaled by 1e300 instead is
    an ordinary row and is served.  The plain fp64 solve serves both."""
    n = 100003
    s = synth.system(78, n)
    t = dict(s, b=s["b"].copy())
    t["b"][n // 2] = 1e300
    _, info = solve(t, flags=ROUTES[route])
    assert info["status_name"] == "TPS_ERR_RANGE", info
    x, info = solve(t, dtype="f64", flags=ROUTES[route])
    assert info["status"] == 0
    assert_matches(t, x)
    rows = np.ones(n)
    rows[n // 2] = 1e300
    u = scaled(s, rows=rows)
    x, info = solve(u, flags=ROUTES[route])
    assert info["status"] == 0, info
    assert_matches(u, x)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_non_finite_x_is_reported_in_every_dtype(dtype):
    n = 100003
    s = synth.system(79, n)
    s["d"][n // 4] = np.nan
    tdt = torch.float64
    if dtype == "f32":
        s, tdt = synth.to_f32(s), torch.float32
    a, b, c, d = (torch.as_tensor(s[k]).to("cuda", tdt) for k in "abcd")
    x = torch.empty_like(b)
    plan = binding.Plan(n, dtype=dtype)
    plan.solve(a, b, c, d, x)
    assert plan.query()["status_name"] == "TPS_ERR_RANGE"


def test_one_warp_solve_range():
    for n in (1, 2, 40, 64):
        s = synth.system(80 + n, n)
        x, info = solve(scaled(s, rows=2.0 ** -700))
        assert info["status"] == 0
        assert_matches(s, x)
        _, info = solve(scaled(s, rhs=2.0 ** -100))
        assert info["status_name"] == "TPS_ERR_RANGE"


@pytest.mark.parametrize("low", [-80, -100])
def test_batched_range_is_per_system(low):
    """One packed system with d scaled by 2^low among ordinary ones: at -80
    every system matches; at -100 that system is reported."""
    sizes = [700, 5, 64, 30000, 1, 4097, 129]
    off = synth.offsets_from_sizes(sizes)
    n = int(off[-1])
    s = synth.system(81, n, offsets=off)
    s["d"][off[3]:off[4]] *= 2.0 ** low
    a, b, c, d = (dev(s[k]) for k in "abcd")
    x = torch.empty_like(b)
    plan = binding.Plan(n, dtype="f64_df", batch_max=len(sizes), m=32)
    plan.solve_batched(torch.as_tensor(off, device="cuda"), a, b, c, d, x, host_offsets=off)
    info = plan.query()
    if low == -100:
        assert info["status_name"] == "TPS_ERR_RANGE"
        return
    assert info["status"] == 0
    xs = x.cpu().numpy()
    ref = oracle.thomas_batched(off, s["a"], s["b"], s["c"], s["d"])
    for i in range(len(sizes)):
        lo, hi = off[i], off[i + 1]
        assert oracle.rel_forward_error(xs[lo:hi], ref[lo:hi]) <= FWD


def test_host_pipeline_range():
    n = 1 << 20
    s = synth.system(82, n)
    plan = binding.Plan(n, dtype="f64_df", residency="host", streams=4)
    for rhs, want in ((2.0 ** -80, "TPS_OK"), (2.0 ** -100, "TPS_ERR_RANGE")):
        t = scaled(s, rhs=rhs)
        a, b, c, d = (torch.as_tensor(t[k]).pin_memory() for k in "abcd")
        x = torch.empty(n, dtype=torch.float64).pin_memory()
        plan.solve_host_async(a, b, c, d, x)
        torch.cuda.synchronize()
        assert plan.query()["status_name"] == want
        if want == "TPS_OK":
            assert_matches(t, x.numpy())


def test_windowed_solve_range():
    n = 1 << 20
    s = synth.system(83, n)
    plan = binding.Plan(n, dtype="f64_df", flags=binding.TRUNCATE)
    for rows, rhs, want in ((2.0 ** -600, 1.0, "TPS_OK"), (1.0, 2.0 ** -100, "TPS_ERR_RANGE")):
        t = scaled(s, rows=rows, rhs=rhs)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        plan.solve(*(dev(t[k]) for k in "abcd"), x)
        assert plan.query()["status_name"] == want
        if want == "TPS_OK":
            assert_matches(s, x.cpu().numpy())


def test_noalloc_range():
    L = binding.lib()
    f = L.tps_solve_noalloc
    P = ctypes.c_void_p
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, P, P, P, P, P]
    f.restype = ctypes.c_int
    n = 100003
    s = synth.system(84, n)
    for rhs, want in ((2.0 ** -80, 0), (2.0 ** -100, 8), (2.0 ** 80, 0)):
        t = scaled(s, rows=2.0 ** 300, rhs=rhs)
        a, b, c, d = (dev(t[k]) for k in "abcd")
        x = torch.empty_like(b)
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert f(binding.DTYPES["f64_df"], n, *(P(v.data_ptr()) for v in (a, b, c, d, x)),
                 P(st.data_ptr()), P(torch.cuda.current_stream().cuda_stream)) == 0
        torch.cuda.synchronize()
        assert st.item() == want
        if want == 0:
            assert_matches(t, x.cpu().numpy())


@pytest.mark.parametrize("e,want", [(-40, "TPS_OK"), (40, "TPS_OK"), (-100, "TPS_ERR_RANGE")])
def test_mixed_refinement_range(e, want):
    """The mixed solve's first fp32 elimination carries the same range codes:
    a right-hand side below what it can represent is reported instead of
    'converging' to x = 0; inside the range it refines to the fp64 bar."""
    n = 100003
    s = scaled(synth.system(85, n), rhs=2.0 ** e)
    x, info = solve(s, dtype="mixed")
    assert info["status_name"] == want, info
    if want == "TPS_OK":
        assert_matches(s, x)
