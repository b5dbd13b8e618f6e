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
