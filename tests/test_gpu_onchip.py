"""The single-launch on-chip solve (one cooperative launch: each CTA
eliminates its rows in shared memory, one grid barrier, the CTA interface
system by parallel cyclic reduction, recovery on chip) against the CPU
oracle, at its capacity edges, as the Stage 2 of larger solves, inside a
captured CUDA graph, and with its barrier wait made to run out."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2501_05938_gb300 import binding, synth

pytestmark = pytest.mark.gpu

F64_FWD, F64_RES = 1e-10, 1e-12
F32_FWD, F32_RES = 1e-5, 1e-5
SMS = 152
CAP = {"f64": SMS * 256 * 23, "f64_df": SMS * 256 * 23, "f32": SMS * 256 * 47,
       "mixed": SMS * 256 * 23}


def solve(plan, s, tdt):
    a, b, c, d = (torch.as_tensor(np.ascontiguousarray(s[k])).to(device="cuda", dtype=tdt)
                  for k in "abcd")
    x = torch.full_like(b, float("nan"))
    plan.solve(a, b, c, d, x)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64), plan.query()


def check(dtype, n, seed, expect_onchip):
    s = synth.system(seed, n)
    tdt = torch.float64
    if dtype == "f32":
        s, tdt = synth.to_f32(s), torch.float32
    x, info = solve(binding.Plan(n, dtype=dtype), s, tdt)
    assert info["status"] == 0
    assert info["onchip"] == expect_onchip, info
    a, b, c, d = (np.asarray(s[k], dtype=np.float64) for k in "abcd")
    ref = oracle.thomas(a, b, c, d)
    fwd, res = (F32_FWD, F32_RES) if dtype == "f32" else (F64_FWD, F64_RES)
    assert oracle.rel_forward_error(x, ref) <= fwd
    assert oracle.rel_residual(a, b, c, d, x) <= res
    return x


@pytest.mark.skipif(torch.cuda.is_available() and
                    torch.cuda.get_device_properties(0).multi_processor_count != SMS,
                    reason="capacity figures assume 152 SMs")
@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32", "mixed"])
def test_capacity_edges(dtype):
    cap = CAP[dtype]
    # the largest system, one more row (a merged one-row tail), then too big
    check(dtype, cap, 11, 1)
    check(dtype, cap + 1, 12, 1)
    check(dtype, cap + 2, 13, 2)


@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32"])
@pytest.mark.parametrize("n", [65, 66, 100, 769, 770, 1000, 4097, 65537, 300001])
def test_small_and_mid_sizes(dtype, n):
    check(dtype, n, 20 + n, 1)


def test_matches_the_multi_launch_path():
    n = 500001
    s = synth.system(5, n)
    xo, io = solve(binding.Plan(n, dtype="f64"), s, torch.float64)
    xm, im = solve(binding.Plan(n, dtype="f64", flags=binding.NO_ONCHIP), s, torch.float64)
    assert io["onchip"] == 1 and im["onchip"] == 0
    assert oracle.rel_forward_error(xo, xm) <= 1e-14


@pytest.mark.parametrize("dtype", ["f64_df", "f64"])
def test_reduced_system_on_chip(dtype):
    n = (1 << 22) + 3
    g = synth.system_device(31, n)
    for flags in (0, binding.GRAPH):
        x = torch.empty_like(g["b"])
        plan = binding.Plan(n, dtype=dtype, m=128, flags=flags)
        for _ in range(2):  # graph: capture, then replay
            x.zero_()
            plan.solve(g["a"], g["b"], g["c"], g["d"], x)
            torch.cuda.synchronize()
            info = plan.query()
            assert info["status"] == 0 and info["onchip"] == 2
            err = ((x - g["x_true"]).abs().max() / g["x_true"].abs().max()).item()
            assert err <= 1e-12


def test_batched_reduced_system_on_chip():
    sizes = synth.batch_sizes(77, 64, 10, 16)
    off = synth.offsets_from_sizes(sizes)
    n = int(off[-1])
    s = synth.system(78, n, offsets=off)
    a, b, c, d = (torch.as_tensor(s[k]).cuda() for k in "abcd")
    x = torch.empty_like(b)
    plan = binding.Plan(n, dtype="f64_df", batch_max=64, m=32)
    plan.solve_batched(torch.as_tensor(off, device="cuda"), a, b, c, d, x, host_offsets=off)
    torch.cuda.synchronize()
    info = plan.query()
    assert info["status"] == 0 and info["onchip"] == 2
    ref = oracle.thomas_batched(off, s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x.cpu().numpy(), ref) <= F64_FWD


def test_barrier_timeout_is_reported_and_the_gpu_stays_usable(monkeypatch):
    n = 100003
    s = synth.system(3, n)
    monkeypatch.setenv("TPS_TEST_ONCHIP_TIMEOUT", "1")
    plan = binding.Plan(n, dtype="f64")
    monkeypatch.delenv("TPS_TEST_ONCHIP_TIMEOUT")
    _, info = solve(plan, s, torch.float64)
    assert info["status_name"] == "TPS_ERR_TIMEOUT"
    # the context survives: the next solve on a normal plan is correct
    check("f64", n, 3, 1)
