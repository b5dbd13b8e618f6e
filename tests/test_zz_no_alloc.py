"""tps_solve_noalloc: the allocation-free solve for callers that may not call
cudaMalloc (a framework allocator that owns all device memory, a fixed
device-memory budget, latency-critical loops).  Its result must agree with the
ordinary plan-based tps_solve and with the CPU oracle, and two calls in a row
must both be right even though they share the library's fixed scratch array.
Both of its routes are run: the single-launch on-chip solve it takes for
every accepted size on a GB300, and the level-by-level route it keeps for
devices where that launch does not fit (forced here by a test switch).  This
file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2501_05938_gb300 import binding, synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f64_df": 1e-10, "f32": 1e-5}
# against the fp64 oracle: (forward error, residual); fp32 on the fp32-rounded inputs
ORACLE_TOL = {"f64": (1e-10, 1e-12), "f64_df": (1e-10, 1e-12), "f32": (1e-5, 1e-5)}


def noalloc_fn():
    L = binding.lib()
    f = L.tps_solve_noalloc
    P = ctypes.c_void_p
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, P, P, P, P, P]
    f.restype = ctypes.c_int
    return f


def rel(x, y):
    x, y = x.double(), y.double()
    return ((x - y).abs().max() / y.abs().max()).item()


def check_two_calls(dtype):
    """Two calls in a row (the largest size, then a ragged one), each against
    the plan-based tps_solve on its level-by-level route and the oracle."""
    f = noalloc_fn()
    tdt = torch.float32 if dtype == "f32" else torch.float64
    stream = torch.cuda.current_stream()
    for seed, n in ((21, 262144), (22, 100003)):
        s = synth.system(seed, n)
        if dtype == "f32":
            s = synth.to_f32(s)
        a, b, c, d = (torch.as_tensor(s[k]).to("cuda", tdt) for k in "abcd")
        x_ref = torch.empty_like(b)
        binding.Plan(n, dtype=dtype, m=64, m_reduced=32,
                     flags=binding.NO_ONCHIP).solve(a, b, c, d, x_ref)
        x = torch.full_like(b, float("nan"))
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = f(binding.DTYPES[dtype], n, *(ctypes.c_void_p(t.data_ptr()) for t in (a, b, c, d, x)),
               ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert st.item() == 0
        assert rel(x, x_ref) <= TOL[dtype]
        s64 = {k: np.asarray(s[k], dtype=np.float64) for k in "abcd"}
        ref = oracle.thomas(s64["a"], s64["b"], s64["c"], s64["d"])
        xs = x.cpu().numpy().astype(np.float64)
        fwd, res = ORACLE_TOL[dtype]
        assert oracle.rel_forward_error(xs, ref) <= fwd
        assert oracle.rel_residual(s64["a"], s64["b"], s64["c"], s64["d"], xs) <= res


@pytest.mark.parametrize("dtype", ["f64_df", "f64", "f32"])
def test_noalloc_matches_tps_solve_on_two_calls(dtype):
    check_two_calls(dtype)


@pytest.mark.parametrize("dtype", ["f64_df", "f64", "f32"])
def test_noalloc_level_route_on_two_calls(dtype, monkeypatch):
    # the route whose reduced systems and checkpoints live in the shared
    # scratch array; the switch is read on every call
    monkeypatch.setenv("TPS_TEST_NOALLOC_LEVELS", "1")
    check_two_calls(dtype)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    f = noalloc_fn()
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    too_big = 262144 + 1
    assert f(0, too_big, p, p, p, p, p, None, None) == 1  # TPS_ERR_INVALID_ARG
    assert f(2, 10, p, p, p, p, p, None, None) == 1       # mixed precision is not served
