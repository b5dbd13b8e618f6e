"""TPS_TRUNCATE (the windowed, truncated decoupling -- an approximation, not
the paper's method) against the truncated-decoupling oracle element by
element, its error bound against the oracle's, the tolerance check, the
chosen parameters against the exact solution, and argument checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import truncated as TR
from paper_2501_05938_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def run(plan, s, tdt=torch.float64):
    a, b, c, d = (torch.as_tensor(np.ascontiguousarray(s[k])).to(device="cuda", dtype=tdt)
                  for k in "abcd")
    x = torch.full_like(b, float("nan"))
    plan.solve(a, b, c, d, x)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64), plan.query()


@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32"])
@pytest.mark.parametrize("n,R,h", [(65, 64, 4), (1000, 96, 16), (20001, 512, 2), (3000, 2, 2),
                                   (70001, 1024, 384), (300001, 1584, 104), (65, 1584, 104)])
def test_matches_the_truncation_oracle(dtype, n, R, h):
    s = synth.system(400 + n + h, n)
    tdt = torch.float64
    if dtype == "f32":
        s, tdt = synth.to_f32(s), torch.float32
    a, b, c, d = (np.asarray(s[k], dtype=np.float64) for k in "abcd")
    xr, br = TR.truncated(a, b, c, d, R, h)
    plan = binding.Plan(n, dtype=dtype, m=R, m_reduced=h, tol=1.0, flags=binding.TRUNCATE)
    x, info = run(plan, s, tdt)
    assert info["m"] == R and info["m_reduced"] == h
    tol = 1e-5 if dtype == "f32" else 1e-11
    # the same windows, solved on the device: agreement up to rounding
    assert oracle.rel_forward_error(x, xr) <= tol
    # the device's bound is the oracle's, rounded up (fp32 with margins;
    # bounds below the fp32 range come out as 0)
    bmax = float(np.max(br))
    if bmax > 1e-30:
        assert bmax * (1 - 1e-4) <= info["last_correction"] <= bmax * 1.01
    else:
        assert info["last_correction"] <= 1e-30
    expect = "TPS_OK" if bmax <= 1.0 else "TPS_ERR_NO_CONVERGENCE"
    assert info["status_name"] == expect


# R + 2 h = 32 mb: the one-warp windows (mb = 8, 16, 56, 64, 256; a clipped
# one-row block at the end for n = 1865 and 300001; one window for n = 65, 1000)
WARP_CASES = [(65, 2040, 4), (1000, 2040, 4), (1865, 1840, 104), (100003, 1840, 104),
              (262144, 1840, 104), (300001, 1840, 104), (70001, 240, 8), (20003, 480, 16),
              (70001, 1024, 384), (1_000_003, 7984, 104), (4099, 1744, 152)]


@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32"])
@pytest.mark.parametrize("n,R,h", WARP_CASES)
def test_warp_windows_match_the_truncation_oracle(dtype, n, R, h):
    """The one-warp windows (each lane a block of mb rows, the partition
    method inside the warp): the oracle's windows element by element, its
    bound, and the same bits on a second solve (the relation buffer is
    discarded from L2 after each use)."""
    s = synth.system(700 + n + h, n)
    tdt = torch.float64
    if dtype == "f32":
        s, tdt = synth.to_f32(s), torch.float32
    a, b, c, d = (np.asarray(s[k], dtype=np.float64) for k in "abcd")
    xr, br = TR.truncated(a, b, c, d, R, h)
    plan = binding.Plan(n, dtype=dtype, m=R, m_reduced=h, tol=1.0, flags=binding.TRUNCATE)
    x, info = run(plan, s, tdt)
    x2, info2 = run(plan, s, tdt)
    np.testing.assert_array_equal(x2, x)
    tol = 1e-5 if dtype == "f32" else 1e-11
    assert oracle.rel_forward_error(x, xr) <= tol
    bmax = float(np.max(br))
    if bmax > 1e-30:
        assert bmax * (1 - 1e-4) <= info["last_correction"] <= bmax * 1.01
    else:
        assert info["last_correction"] <= 1e-30
    expect = "TPS_OK" if bmax <= 1.0 else "TPS_ERR_NO_CONVERGENCE"
    assert info["status_name"] == expect
    if dtype != "f32" and bmax <= 1e-12:
        ref = oracle.thomas(a, b, c, d)
        assert oracle.rel_forward_error(x, ref) <= 1e-10
        assert oracle.rel_residual(a, b, c, d, x) <= 1e-12


def test_bound_over_tolerance_is_reported():
    n = 20000
    s = synth.system(9, n)
    plan = binding.Plan(n, dtype="f64_df", m=512, m_reduced=2, tol=1e-12,
                        flags=binding.TRUNCATE)
    _, info = run(plan, s)
    assert info["status_name"] == "TPS_ERR_NO_CONVERGENCE"
    assert info["last_correction"] > 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f64_df"])
def test_chosen_parameters_meet_the_tolerance(dtype):
    n = 1_000_003
    s = synth.system(17, n)
    plan = binding.Plan(n, dtype=dtype, flags=binding.TRUNCATE)
    x, info = run(plan, s)
    assert info["status"] == 0 and info["last_correction"] <= 1e-12
    assert info["m"] % 2 == 0 and info["m_reduced"] % 2 == 0
    # the default windows are one-warp windows of 32 blocks of 256 rows
    assert info["m"] + 2 * info["m_reduced"] == 8192
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x, ref) <= 1e-10
    assert oracle.rel_residual(s["a"], s["b"], s["c"], s["d"], x) <= 1e-12


def test_weakly_dominant_system_is_flagged():
    # ratio 1.01: q ~ 0.99, a 104-row halo cannot meet 1e-12
    n = 100000
    s = synth.system(5, n, kind=synth.KIND_RATIO, ratio=1.01)
    plan = binding.Plan(n, dtype="f64_df", flags=binding.TRUNCATE)
    _, info = run(plan, s)
    assert info["status_name"] == "TPS_ERR_NO_CONVERGENCE"


def test_arguments():
    n = 1000
    with pytest.raises(binding.TpsError):
        binding.Plan(n, dtype="f64", m=101, flags=binding.TRUNCATE)  # odd window
    with pytest.raises(binding.TpsError):
        binding.Plan(n, dtype="f64", m=1500, m_reduced=200, flags=binding.TRUNCATE)  # > 1792
    with pytest.raises(binding.TpsError):
        binding.Plan(n, dtype="mixed", flags=binding.TRUNCATE)
    with pytest.raises(binding.TpsError):
        binding.Plan(n, dtype="f64", residency="host", flags=binding.TRUNCATE)
    plan = binding.Plan(n, dtype="f64", batch_max=4, flags=binding.TRUNCATE)
    off = np.array([0, 500, 1000], dtype=np.int64)
    t = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.TpsError):
        plan.solve_batched(torch.as_tensor(off, device="cuda"), t, t, t, t, torch.empty_like(t),
                           host_offsets=off)


@pytest.mark.slow
def test_full_size_against_the_exact_oracle():
    n = 1 << 27
    g = synth.system_device(1002, n)
    x = torch.empty_like(g["b"])
    plan = binding.Plan(n, dtype="f64_df", flags=binding.TRUNCATE)
    plan.solve(g["a"], g["b"], g["c"], g["d"], x)
    torch.cuda.synchronize()
    info = plan.query()
    assert info["status"] == 0 and info["last_correction"] <= 1e-12
    a, b, c, d = (g[k].cpu().numpy() for k in "abcd")
    del g
    ref = oracle.thomas(a, b, c, d)
    xs = x.cpu().numpy()
    assert oracle.rel_forward_error(xs, ref) <= 1e-10
    assert oracle.rel_residual(a, b, c, d, xs) <= 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f64_df"])
@pytest.mark.parametrize("R,h", [(1576, 104), (1840, 104)])  # one-CTA, one-warp windows
@pytest.mark.parametrize("rows", [2.0 ** -600, 2.0 ** 300])
def test_bound_is_scale_free(dtype, R, h, rows):
    """Every row multiplied by the same power of two: x is unchanged, and so
    is each window's bound (a ratio of couplings to diagonals), also far
    outside binary32's range, where a bound computed from fp32 copies of the
    entries would under- or overflow."""
    n = 100003
    s = synth.system(88, n)
    t = {k: np.asarray(s[k], dtype=np.float64) * rows for k in "abcd"}
    plan = binding.Plan(n, dtype=dtype, m=R, m_reduced=h, tol=1.0, flags=binding.TRUNCATE)
    x0, i0 = run(plan, s)
    x1, i1 = run(plan, t)
    assert i0["status"] == 0 and i1["status"] == 0, (i0, i1)
    assert oracle.rel_forward_error(x1, x0) <= 1e-14
    assert 0.0 < i0["last_correction"] < 1e-12
    assert abs(i1["last_correction"] - i0["last_correction"]) <= 1e-5 * i0["last_correction"]
