"""Mixed-precision refinement (fp32 partition elimination, fp64 residual and
update) against the fp64 Thomas oracle, on the dominance ratios of the
refinement workload (b = r (|a| + |c|), r in {1.01, 1.1, 2.0})."""
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import refine as orefine
from paper_2501_05938_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def solve_mixed(s, n, **kw):
    a, b, c, d = (torch.as_tensor(s[k]).cuda() for k in "abcd")
    x = torch.empty_like(b)
    plan = binding.Plan(n, dtype="mixed", **kw)
    plan.solve(a, b, c, d, x)
    torch.cuda.synchronize()
    return x.cpu().numpy(), plan.query()


@pytest.mark.parametrize("ratio", [1.01, 1.1, 2.0])
@pytest.mark.parametrize("n", [300001, 65])
def test_refinement_reaches_fp64_accuracy(ratio, n):
    s = synth.system(50 + n, n, kind=synth.KIND_RATIO, ratio=ratio)
    x, info = solve_mixed(s, n, m=64)
    assert info["status"] == 0, info
    assert 1 <= info["iterations"] <= 10
    assert info["last_correction"] <= 1e-12
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x, ref) <= 1e-10
    assert oracle.rel_residual(s["a"], s["b"], s["c"], s["d"], x) <= 1e-12
    # the same algorithm step by step on the CPU needs a similar count
    _, it_ref, ok = orefine.refine(s["a"], s["b"], s["c"], s["d"], tol=1e-12)
    assert ok and abs(info["iterations"] - it_ref) <= 2


def test_paper_generator_converges_in_few_iterations():
    n = 1 << 20
    s = synth.system(3, n)
    x, info = solve_mixed(s, n)
    assert info["status"] == 0 and info["iterations"] <= 3
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x, ref) <= 1e-10


def test_iteration_cap_reports_no_convergence():
    n = 100000
    s = synth.system(4, n, kind=synth.KIND_RATIO, ratio=1.01)
    _, info = solve_mixed(s, n, max_iters=1, tol=1e-30)
    assert info["status_name"] == "TPS_ERR_NO_CONVERGENCE"
    assert info["iterations"] == 1


def test_batched_refinement():
    sizes = synth.batch_sizes(1005, 64, 10, 14)
    off = synth.offsets_from_sizes(sizes)
    n = int(off[-1])
    s = synth.system(1005, n, kind=synth.KIND_RATIO, ratio=1.1, offsets=off)
    a, b, c, d = (torch.as_tensor(s[k]).cuda() for k in "abcd")
    x = torch.empty_like(b)
    plan = binding.Plan(n, dtype="mixed", batch_max=len(sizes))
    plan.solve_batched(torch.as_tensor(off, device="cuda"), a, b, c, d, x, host_offsets=off)
    torch.cuda.synchronize()
    info = plan.query()
    assert info["status"] == 0 and info["iterations"] >= 1
    ref = oracle.thomas_batched(off, s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x.cpu().numpy(), ref) <= 1e-10


@pytest.mark.slow
@pytest.mark.parametrize("ratio", [1.01, 2.0])
def test_full_size_refinement(ratio):
    """n = 2^27 single system and 1024 systems with n_i log-uniform in
    [2^10, 2^18] (the refinement workload)."""
    n = 1 << 27
    g = synth.system_device(1005, n, kind=synth.KIND_RATIO, ratio=ratio)
    x = torch.empty_like(g["b"])
    plan = binding.Plan(n, dtype="mixed")
    plan.solve(g["a"], g["b"], g["c"], g["d"], x)
    torch.cuda.synchronize()
    info = plan.query()
    assert info["status"] == 0, info
    h = {k: g[k].cpu().numpy() for k in "abcd"}
    del g
    ref = oracle.thomas(h["a"], h["b"], h["c"], h["d"])
    assert oracle.rel_forward_error(x.cpu().numpy(), ref) <= 1e-10
    del x
    sizes = synth.batch_sizes(1006, 1024, 10, 18)
    off = synth.offsets_from_sizes(sizes)
    nb = int(off[-1])
    g = synth.system_device(1006, nb, kind=synth.KIND_RATIO, ratio=ratio, offsets=off)
    x = torch.empty_like(g["b"])
    plan = binding.Plan(nb, dtype="mixed", batch_max=1024)
    plan.solve_batched(torch.as_tensor(off, device="cuda"), g["a"], g["b"], g["c"], g["d"], x,
                       host_offsets=off)
    torch.cuda.synchronize()
    assert plan.query()["status"] == 0
    h = {k: g[k].cpu().numpy() for k in "abcd"}
    ref = oracle.thomas_batched(off, h["a"], h["b"], h["c"], h["d"])
    assert oracle.rel_forward_error(x.cpu().numpy(), ref) <= 1e-10


# The corrections run fused into level 0's sweeps (Stage 1 forms the fp64
# residual from the rows and x, Stage 3 adds delta to x in place) wherever
# the system is solved level by level; TPS_TEST_UNFUSED_REFINE=1 at plan
# time keeps the separate residual / solve / update passes.  Both against
# the oracle, and against each other.
def solve_mixed_plan(s, n, monkeypatch, unfused, offsets=None, **kw):
    if unfused:
        monkeypatch.setenv("TPS_TEST_UNFUSED_REFINE", "1")
    else:
        monkeypatch.delenv("TPS_TEST_UNFUSED_REFINE", raising=False)
    a, b, c, d = (torch.as_tensor(s[k]).cuda() for k in "abcd")
    x = torch.empty_like(b)
    if offsets is None:
        plan = binding.Plan(n, dtype="mixed", **kw)
        plan.solve(a, b, c, d, x)
    else:
        plan = binding.Plan(n, dtype="mixed", batch_max=len(offsets) - 1, **kw)
        plan.solve_batched(torch.as_tensor(offsets, device="cuda"), a, b, c, d, x,
                           host_offsets=offsets)
    torch.cuda.synchronize()
    info = plan.query()
    monkeypatch.delenv("TPS_TEST_UNFUSED_REFINE", raising=False)
    return x.cpu().numpy(), info


NO_OC = binding.NO_ONCHIP
FUSED_CASES = [
    # (n, m, flags, ratio): several tiles and a ragged tail (the single-launch
    # on-chip solve off, so that level 0 runs as separate sweeps); m = 51
    # takes the element-by-element loads (m not a multiple of the 16-byte
    # vector); the tail block of m + 1 rows; a size the on-chip solve does
    # not take (if it did, the corrections would run as separate passes)
    (300001, 64, NO_OC, 1.01),
    (300001, 64, NO_OC, 2.0),
    (123457, 51, NO_OC, 1.1),
    (5000, 16, NO_OC, 1.01),
    (128 * 40 + 129, 128, NO_OC, 1.1),
    (1 << 23, 128, 0, 1.01),
]


@pytest.mark.parametrize("n,m,flags,ratio", FUSED_CASES)
def test_fused_refinement_against_oracle_and_unfused(n, m, flags, ratio, monkeypatch):
    s = synth.system(70 + n % 97, n, kind=synth.KIND_RATIO, ratio=ratio)
    xf, inf_f = solve_mixed_plan(s, n, monkeypatch, False, m=m, flags=flags)
    xu, inf_u = solve_mixed_plan(s, n, monkeypatch, True, m=m, flags=flags)
    assert inf_f["status"] == 0 and inf_u["status"] == 0, (inf_f, inf_u)
    assert inf_f["refine_fused"] == (inf_f["onchip"] != 1) and not inf_u["refine_fused"]
    if flags & NO_OC:
        assert inf_f["refine_fused"]
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    for x in (xf, xu):
        assert oracle.rel_forward_error(x, ref) <= 1e-10
        assert oracle.rel_residual(s["a"], s["b"], s["c"], s["d"], x) <= 1e-12
    # the two differ only in the rounding of the residual's three products
    assert abs(inf_f["iterations"] - inf_u["iterations"]) <= 1
    assert oracle.rel_forward_error(xf, xu) <= 1e-13
    assert inf_f["last_correction"] <= 1e-12


def test_fused_refinement_on_packed_systems(monkeypatch):
    """Couplings cut at every system boundary: the residual of a system's
    first and last row must not read its neighbours' x."""
    sizes = synth.batch_sizes(2024, 200, 3, 14)
    off = synth.offsets_from_sizes(sizes)
    n = int(off[-1])
    s = synth.system(2024, n, kind=synth.KIND_RATIO, ratio=1.01, offsets=off)
    xf, inf_f = solve_mixed_plan(s, n, monkeypatch, False, offsets=off, m=32, flags=NO_OC)
    xu, inf_u = solve_mixed_plan(s, n, monkeypatch, True, offsets=off, m=32, flags=NO_OC)
    assert inf_f["status"] == 0 and inf_u["status"] == 0
    assert inf_f["refine_fused"] and not inf_u["refine_fused"]
    ref = oracle.thomas_batched(off, s["a"], s["b"], s["c"], s["d"])
    for x in (xf, xu):
        assert oracle.rel_forward_error(x, ref) <= 1e-10
    assert abs(inf_f["iterations"] - inf_u["iterations"]) <= 1


def test_onchip_route_keeps_separate_passes(monkeypatch):
    n = 65536
    s = synth.system(77, n, kind=synth.KIND_RATIO, ratio=1.1)
    x, info = solve_mixed_plan(s, n, monkeypatch, False)
    assert info["status"] == 0
    assert info["refine_fused"] == (info["onchip"] != 1)
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x, ref) <= 1e-10


def test_fused_refinement_iteration_cap(monkeypatch):
    n = 100000
    s = synth.system(4, n, kind=synth.KIND_RATIO, ratio=1.01)
    _, info = solve_mixed_plan(s, n, monkeypatch, False, m=64, flags=NO_OC,
                               max_iters=1, tol=1e-30)
    assert info["refine_fused"]
    assert info["status_name"] == "TPS_ERR_NO_CONVERGENCE"
    assert info["iterations"] == 1
