"""GPU parity: libtps through its C ABI against the CPU oracle.

Tolerances
  fp64 paths (TPS_F64, TPS_F64_DF): relative forward error <= 1e-10 against
  the fp64 Thomas oracle and relative residual <= 1e-12, the bar the solver
  is specified to.  For these generators kappa_inf(A) <= 6, so a backward-
  stable fp64 solve sits near 1e-15; the double-float path near 1e-13.
  fp32 path (TPS_F32): against the fp64 oracle on the fp32-rounded inputs,
  relative forward error <= 1e-5 and residual <= 1e-5 (kappa 6 times a few
  hundred binary32 roundings of 6e-8).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2501_05938_gb300 import binding, synth

pytestmark = pytest.mark.gpu

F64_FWD, F64_RES = 1e-10, 1e-12
F32_FWD, F32_RES = 1e-5, 1e-5


def dev(v, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(v)).to(device="cuda", dtype=dtype)


def run(plan, s, dtype=torch.float64):
    a, b, c, d = (dev(s[k], dtype) for k in "abcd")
    x = torch.empty_like(b)
    plan.solve(a, b, c, d, x)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64), plan.query()


def test_device_generator_is_bit_identical_to_numpy():
    for n, off in ((100003, None), (5000, synth.offsets_from_sizes([1, 2, 3, 1000, 3994]))):
        h = synth.system(1002, n, offsets=off)
        g = synth.system_device(1002, n, offsets=off)
        for k in ("a", "b", "c", "d", "x_true"):
            np.testing.assert_array_equal(g[k].cpu().numpy(), h[k])
        h = synth.system(77, n, kind=synth.KIND_RATIO, ratio=1.01, offsets=off)
        g = synth.system_device(77, n, kind=synth.KIND_RATIO, ratio=1.01, offsets=off)
        for k in ("a", "b", "c", "d", "x_true"):
            np.testing.assert_array_equal(g[k].cpu().numpy(), h[k])


CASES = [(1, 32), (2, 32), (3, 2), (63, 8), (64, 32), (65, 32), (65, 2), (100, 3), (1000, 10),
         (4097, 8), (4096, 33), (65536, 256), (100003, 32), (100003, 1024), (262145, 64),
         (1 << 20, 32), ((1 << 20) + 7, 100)]


@pytest.mark.parametrize("onchip", [True, False])
@pytest.mark.parametrize("dtype", ["f64", "f64_df"])
@pytest.mark.parametrize("n,m", CASES)
def test_fp64_paths_match_oracle(dtype, n, m, onchip):
    """Both routes: the single-launch on-chip solve where the system fits,
    and the multi-launch levels (TPS_NO_ONCHIP)."""
    s = synth.system(1000 + n, n)
    plan = binding.Plan(n, dtype=dtype, m=m, flags=0 if onchip else binding.NO_ONCHIP)
    x, info = run(plan, s)
    assert info["status"] == 0
    if not onchip:
        assert info["onchip"] == 0
    elif n > 64:
        assert info["onchip"] in (1, 2)
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    fwd = oracle.rel_forward_error(x, ref)
    res = oracle.rel_residual(s["a"], s["b"], s["c"], s["d"], x)
    assert fwd <= F64_FWD, fwd
    assert res <= F64_RES, res
    if dtype == "f64":  # the plain solve keeps fp64 accuracy (kappa <= 6)
        assert fwd <= 1e-14 and res <= 1e-15, (fwd, res)


@pytest.mark.parametrize("m", [16, 24, 64])
@pytest.mark.parametrize("tail", [0, 1, 5, 9])
@pytest.mark.parametrize("dtype", ["f64_df", "f32"])
def test_chunk_kinds_at_block_and_warp_edges(m, tail, dtype):
    """Block counts that end a warp exactly, one block into a warp, or one
    short of it, with a last block of m, m + 1 (merged one-row tail), or a
    few rows: the unrolled first/last-chunk paths and the row-by-row path
    meet at these edges."""
    tdt = torch.float32 if dtype == "f32" else torch.float64
    fwd_tol, res_tol = (F32_FWD, F32_RES) if dtype == "f32" else (F64_FWD, F64_RES)
    for p in (32 * 40, 32 * 40 + 1, 32 * 41 - 1):
        n = p * m + tail
        s = synth.system(3000 + n, n)
        if dtype == "f32":
            s = synth.to_f32(s)
        x, info = run(binding.Plan(n, dtype=dtype, m=m, flags=binding.NO_ONCHIP), s, tdt)
        assert info["status"] == 0
        a, b, c, d = (np.asarray(s[k], dtype=np.float64) for k in "abcd")
        ref = oracle.thomas(a, b, c, d)
        assert oracle.rel_forward_error(x, ref) <= fwd_tol, (p, n)
        assert oracle.rel_residual(a, b, c, d, x) <= res_tol, (p, n)


@pytest.mark.parametrize("n,m,mr", [(1 << 16, 256, 4), (1 << 18, 2, 8), (50000, 1000, 1000)])
def test_reduced_block_sizes(n, m, mr):
    """Unusual block sizes on the level-by-level route (the on-chip solve
    would take these sizes whole)."""
    s = synth.system(5 + n, n)
    for dtype in ("f64", "f64_df"):
        plan = binding.Plan(n, dtype=dtype, m=m, m_reduced=mr, flags=binding.NO_ONCHIP)
        x, info = run(plan, s)
        ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
        assert oracle.rel_forward_error(x, ref) <= F64_FWD
        assert info["levels"] >= 1


@pytest.mark.parametrize("n,m", [(65, 16), (4097, 16), (100003, 64), (1 << 20, 32)])
def test_fp32_path_matches_oracle_on_rounded_inputs(n, m):
    s64 = synth.system(2000 + n, n)
    s32 = synth.to_f32(s64)
    plan = binding.Plan(n, dtype="f32", m=m)
    x, info = run(plan, s32, torch.float32)
    assert info["status"] == 0
    a, b, c, d = (s32[k].astype(np.float64) for k in "abcd")
    ref = oracle.thomas(a, b, c, d)
    assert oracle.rel_forward_error(x, ref) <= F32_FWD
    assert oracle.rel_residual(a, b, c, d, x) <= F32_RES


@pytest.mark.parametrize("ratio", [1.01, 1.1, 2.0])
def test_weakly_dominant_systems(ratio):
    n = 300001
    s = synth.system(31, n, kind=synth.KIND_RATIO, ratio=ratio)
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    for dtype in ("f64", "f64_df"):
        x, info = run(binding.Plan(n, dtype=dtype, m=64), s)
        assert info["status"] == 0
        assert oracle.rel_forward_error(x, ref) <= F64_FWD
        assert oracle.rel_residual(s["a"], s["b"], s["c"], s["d"], x) <= F64_RES


def test_zero_pivot_is_reported_not_raised():
    n = 5000
    s = synth.system(3, n)
    s["b"][:] = 0.0
    s["a"][:] = 0.0
    s["c"][:] = 0.0
    for dtype in ("f64", "f64_df"):
        plan = binding.Plan(n, dtype=dtype, m=32)
        _, info = run(plan, s)
        assert info["status_name"] == "TPS_ERR_ZERO_PIVOT"
        # the word is cleared by the query
        assert plan.query()["status"] == 0


def test_workspace_allocation_failure_is_reported():
    # a plan for 2^40 rows needs tens of TB of workspace: cudaMalloc fails, the plan
    # reports TPS_ERR_OOM and nothing is left allocated
    with pytest.raises(binding.TpsError) as ei:
        binding.Plan(1 << 40, dtype="f64")
    assert ei.value.status == 4
    x, info = run(binding.Plan(1000, dtype="f64"), synth.system(1, 1000))  # still usable
    assert info["status"] == 0


@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32"])
@pytest.mark.parametrize("n", [1000, 100003, 1 << 21])
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_diagonal_is_reported(dtype, n, bad):
    s = synth.system(4, n)
    tdt = torch.float64
    if dtype == "f32":
        s, tdt = synth.to_f32(s), torch.float32
    s["b"][n // 3] = bad
    _, info = run(binding.Plan(n, dtype=dtype), s, tdt)
    assert info["status_name"] == "TPS_ERR_ZERO_PIVOT"


@pytest.mark.parametrize("n", [1000, 1 << 21])
def test_double_float_range_is_checked(n):
    # 1e300 is a fine fp64 value but, against a, c, d of order 1 in its row,
    # puts that row's x (about 1e-300) beyond the double-float range: the
    # range is reported, while the plain fp64 solve is exact
    s = synth.system(6, n)
    s["b"][n // 2] = 1e300
    _, info = run(binding.Plan(n, dtype="f64_df"), s)
    assert info["status_name"] == "TPS_ERR_RANGE"
    x, info = run(binding.Plan(n, dtype="f64"), s)
    assert info["status"] == 0
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x, ref) <= F64_FWD


def test_invalid_arguments():
    n = 1000
    plan = binding.Plan(n, dtype="f64")
    a = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    b, c, d, x = (torch.ones(n + 1, dtype=torch.float64, device="cuda") for _ in range(4))
    L = binding.lib()
    st = binding._stream(None)
    P = binding._ptr
    # n above n_max
    assert L.tps_solve(plan.handle, n + 1, P(a), P(b), P(c), P(d), P(x), st) == 1
    # x aliases an input
    assert L.tps_solve(plan.handle, n, P(a), P(b), P(c), P(d), P(a), st) == 1
    # host (pageable) memory given to the device entry point
    h = np.zeros(n)
    hp = binding.ctypes.c_void_p(h.ctypes.data)
    assert L.tps_solve(plan.handle, n, hp, P(b), P(c), P(d), P(x), st) == 1
    # misaligned pointer
    mis = binding.ctypes.c_void_p(a.data_ptr() + 4)
    assert L.tps_solve(plan.handle, n, mis, P(b), P(c), P(d), P(x), st) == 1
    # n = 0 is a no-op
    assert L.tps_solve(plan.handle, 0, P(a), P(b), P(c), P(d), P(x), st) == 0


def test_external_workspace():
    n = 70000
    s = synth.system(8, n)
    plan = binding.Plan(n, dtype="f64_df", m=32, flags=binding.EXTERNAL_WORKSPACE)
    need = plan.workspace_size()
    with pytest.raises(binding.TpsError):  # the workspace must be device memory
        plan.set_workspace(torch.empty(need, dtype=torch.uint8, pin_memory=True))
    with pytest.raises(binding.TpsError):  # and large enough
        plan.set_workspace(torch.empty(need - 256, dtype=torch.uint8, device="cuda"))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    plan.set_workspace(ws)
    x, info = run(plan, s)
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x, ref) <= F64_FWD


@pytest.mark.slow
@pytest.mark.parametrize("dtype", ["f64_df", "f64"])
def test_full_size_single_system(dtype):
    """n = 2^27 (the large single-system workload): every row against the
    serial Thomas oracle run on the host."""
    n = 1 << 27
    g = synth.system_device(1002, n)
    x = torch.empty_like(g["b"])
    plan = binding.Plan(n, dtype=dtype, m=32)
    plan.solve(g["a"], g["b"], g["c"], g["d"], x)
    torch.cuda.synchronize()
    assert plan.query()["status"] == 0
    a, b, c, d = (g[k].cpu().numpy() for k in "abcd")
    del g
    ref = oracle.thomas(a, b, c, d)
    xs = x.cpu().numpy()
    assert oracle.rel_forward_error(xs, ref) <= F64_FWD
    assert oracle.rel_residual(a, b, c, d, xs) <= F64_RES


def pinned(v, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(v)).to(dtype).pin_memory()


@pytest.mark.parametrize("dtype", ["f64", "f64_df"])
@pytest.mark.parametrize("n,m,S,chunk", [(50, 32, 1, 0), (100003, 32, 1, 0), (100003, 32, 4, 0),
                                          (100003, 64, 8, 5000), (262145, 32, 32, 0),
                                          (262145, 1024, 3, 70000)])
def test_host_pipeline_matches_oracle(dtype, n, m, S, chunk):
    s = synth.system(4000 + n, n)
    plan = binding.Plan(n, dtype=dtype, residency="host", m=m, streams=S, chunk=chunk)
    a, b, c, d = (pinned(s[k]) for k in "abcd")
    x = torch.empty(n, dtype=torch.float64).pin_memory()
    stream = torch.cuda.Stream()
    plan.solve_host_async(a, b, c, d, x, stream=stream)
    stream.synchronize()
    info = plan.query()
    assert info["status"] == 0 and info["streams"] == S
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    xs = x.numpy()
    assert oracle.rel_forward_error(xs, ref) <= F64_FWD
    assert oracle.rel_residual(s["a"], s["b"], s["c"], s["d"], xs) <= F64_RES


@pytest.mark.parametrize("flags", [0, binding.ZERO_COPY])
def test_host_autotune_keeps_a_working_stream_and_chunk_choice(flags):
    n = 2_000_003
    s = synth.system(77, n)
    plan = binding.Plan(n, dtype="f64_df", residency="host", streams=2, flags=flags)
    a, b, c, d = (pinned(s[k]) for k in "abcd")
    x = torch.empty(n, dtype=torch.float64).pin_memory()
    stream = torch.cuda.Stream()
    _, ms = plan.autotune(a, b, c, d, x, reps=1, stream=stream)
    info = plan.query()
    assert ms > 0 and info["streams"] in (1, 2, 4, 8, 16, 32)
    assert info["chunk"] in (0, 1 << 22, 1 << 24)
    x.fill_(float("nan"))
    plan.solve_host_async(a, b, c, d, x, stream=stream)
    stream.synchronize()
    assert plan.query()["status"] == 0
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x.numpy(), ref) <= F64_FWD


def host_systems(dtype, n, seeds):
    tdt = torch.float32 if dtype == "f32" else torch.float64
    systems, refs = [], []
    for seed in seeds:
        s = synth.system(seed, n)
        if dtype == "f32":
            s = synth.to_f32(s)
        systems.append(tuple(torch.as_tensor(np.ascontiguousarray(s[k])).to(tdt).pin_memory()
                             for k in "abcd"))
        a, b, c, d = (np.asarray(s[k], dtype=np.float64) for k in "abcd")
        refs.append(oracle.thomas(a, b, c, d))
    return systems, refs, tdt


@pytest.mark.parametrize("dtype,S,flags", [("f64_df", 2, 0), ("f64", 4, binding.GRAPH),
                                           ("f32", 2, binding.ZERO_COPY)])
def test_host_many_overlaps_systems_and_matches_oracle(dtype, S, flags):
    n, count = 300001, 5
    systems, refs, tdt = host_systems(dtype, n, [500 + k for k in range(count)])
    xs = [torch.full((n,), float("nan"), dtype=tdt).pin_memory() for _ in range(count)]
    plan = binding.Plan(n, dtype=dtype, residency="host", streams=S, chunk=1 << 16,
                        flags=binding.HOST_OVERLAP | flags)
    plan.solve_host_many(systems, xs)
    torch.cuda.synchronize()
    info = plan.query()
    assert info["status"] == 0 and info["onchip"] == 0
    tol = F32_FWD if dtype == "f32" else F64_FWD
    for x, ref in zip(xs, refs):
        assert oracle.rel_forward_error(x.numpy().astype(np.float64), ref) <= tol
    # after tps_autotune changes S and chunk, the twin follows
    a, b, c, d = systems[0]
    plan.autotune(a, b, c, d, xs[0], reps=1)
    for x in xs:
        x.fill_(float("nan"))
    plan.solve_host_many(systems, xs)
    torch.cuda.synchronize()
    assert plan.query()["status"] == 0
    for x, ref in zip(xs, refs):
        assert oracle.rel_forward_error(x.numpy().astype(np.float64), ref) <= tol


@pytest.mark.parametrize("n,chunk", [(1, 0), (64, 0), (65, 0), (1000, 100), (70001, 4096)])
def test_host_many_small_and_ragged_sizes(n, chunk):
    systems, refs, tdt = host_systems("f64_df", n, [800 + k for k in range(4)])
    xs = [torch.full((n,), float("nan"), dtype=tdt).pin_memory() for _ in range(4)]
    plan = binding.Plan(n, dtype="f64_df", residency="host", streams=4, chunk=chunk,
                        flags=binding.HOST_OVERLAP)
    plan.solve_host_many(systems, xs)
    torch.cuda.synchronize()
    assert plan.query()["status"] == 0
    for x, ref in zip(xs, refs):
        assert oracle.rel_forward_error(x.numpy(), ref) <= F64_FWD


def test_host_many_zero_copy_from_pageable_memory():
    n = 200003
    plan = binding.Plan(n, dtype="f64", residency="host", streams=2,
                        flags=binding.HOST_OVERLAP | binding.ZERO_COPY)
    if not plan.query()["pageable_ok"]:
        pytest.skip("the device does not access pageable host memory coherently")
    systems, refs, _ = host_systems("f64", n, [900, 901, 902])
    systems = [tuple(t.clone() for t in sy) for sy in systems]  # pageable copies
    xs = [torch.full((n,), float("nan"), dtype=torch.float64) for _ in range(3)]
    plan.solve_host_many(systems, xs)
    torch.cuda.synchronize()
    assert plan.query()["status"] == 0
    for x, ref in zip(xs, refs):
        assert oracle.rel_forward_error(x.numpy(), ref) <= F64_FWD


def test_host_many_reports_the_twins_systems_and_checks_outputs():
    n = 100003
    systems, refs, tdt = host_systems("f64_df", n, [71, 72, 71])
    plan = binding.Plan(n, dtype="f64_df", residency="host", streams=2,
                        flags=binding.HOST_OVERLAP)
    # outputs of systems two apart may be the same buffer
    x0, x1 = (torch.empty(n, dtype=tdt).pin_memory() for _ in range(2))
    plan.solve_host_many(systems, [x0, x1, x0])
    torch.cuda.synchronize()
    assert plan.query()["status"] == 0
    assert oracle.rel_forward_error(x0.numpy(), refs[2]) <= F64_FWD
    assert oracle.rel_forward_error(x1.numpy(), refs[1]) <= F64_FWD
    # a non-finite pivot in system 1 (solved by the twin) reaches the plan's status
    bad = list(systems[1])
    bad[1] = bad[1].clone().pin_memory()
    bad[1][n // 2] = float("nan")
    plan.solve_host_many([systems[0], tuple(bad)], [x0, x1])
    torch.cuda.synchronize()
    assert plan.query()["status_name"] == "TPS_ERR_ZERO_PIVOT"
    assert plan.query()["status"] == 0  # the query resets both status words
    with pytest.raises(binding.TpsError):  # consecutive outputs overlap
        plan.solve_host_many(systems[:2], [x0, x0])
    with pytest.raises(binding.TpsError):  # an output overlaps the next system's input
        plan.solve_host_many(systems[:2], [systems[1][3], x1])
    # system 1's arrays are rejected: system 0 stays enqueued and completes
    x0.fill_(float("nan"))
    dev_b = systems[1][1].cuda()
    with pytest.raises(binding.TpsError):
        plan.solve_host_many([systems[0], (systems[1][0], dev_b, systems[1][2], systems[1][3])],
                             [x0, x1])
    torch.cuda.synchronize()
    assert plan.query()["status"] == 0
    assert oracle.rel_forward_error(x0.numpy(), refs[0]) <= F64_FWD
    plain = binding.Plan(n, dtype="f64_df", residency="host", streams=2)
    with pytest.raises(binding.TpsError):  # the plan has no twin
        plain.solve_host_many(systems[:2], [x0, x1])
    with pytest.raises(binding.TpsError):  # overlap is for host residency
        binding.Plan(n, dtype="f64_df", flags=binding.HOST_OVERLAP)
    plan.solve_host_many([], [])  # nothing to do


def test_host_pipeline_rejects_pageable_and_device_memory():
    n = 1000
    plan = binding.Plan(n, dtype="f64", residency="host", streams=2)
    s = synth.system(1, n)
    pg = [torch.as_tensor(s[k]) for k in "abcd"]  # pageable
    x = torch.empty(n, dtype=torch.float64)
    with pytest.raises(binding.TpsError):
        plan.solve_host_async(*pg, x)
    dv = [t.cuda() for t in pg]
    with pytest.raises(binding.TpsError):
        plan.solve_host_async(*dv, x.cuda())
    # a device plan has no host pipeline
    with pytest.raises(binding.TpsError):
        binding.Plan(n, dtype="f64").solve_host_async(*[t.pin_memory() for t in pg],
                                                       x.pin_memory())


@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32"])
@pytest.mark.parametrize("mem", ["pinned", "pageable"])
@pytest.mark.parametrize("n,m", [(50, 32), (100003, 32), (262145, 128), (65536 * 3 + 1, 64)])
def test_zero_copy_matches_oracle(dtype, mem, n, m):
    """TPS_ZERO_COPY: Stage 1 reads host memory directly and mirrors it,
    Stage 3 writes x straight to host memory."""
    s = synth.system(7000 + n, n)
    tdt = torch.float64
    if dtype == "f32":
        s, tdt = synth.to_f32(s), torch.float32
    plan = binding.Plan(n, dtype=dtype, residency="host", m=m, flags=binding.ZERO_COPY)
    if mem == "pageable" and not plan.query()["pageable_ok"]:
        pytest.skip("the device has no coherent access to pageable host memory")
    host = [torch.as_tensor(np.ascontiguousarray(s[k])).to(tdt) for k in "abcd"]
    x = torch.full((n,), float("nan"), dtype=tdt)
    if mem == "pinned":
        host, x = [t.pin_memory() for t in host], x.pin_memory()
    stream = torch.cuda.Stream()
    plan.solve_host_async(*host, x, stream=stream)
    stream.synchronize()
    assert plan.query()["status"] == 0
    a, b, c, d = (np.asarray(s[k], dtype=np.float64) for k in "abcd")
    ref = oracle.thomas(a, b, c, d)
    xs = x.numpy().astype(np.float64)
    fwd, res = (F32_FWD, F32_RES) if dtype == "f32" else (F64_FWD, F64_RES)
    assert oracle.rel_forward_error(xs, ref) <= fwd
    assert oracle.rel_residual(a, b, c, d, xs) <= res


def test_zero_copy_needs_host_residency_and_host_memory():
    n = 1000
    with pytest.raises(binding.TpsError):
        binding.Plan(n, dtype="f64", flags=binding.ZERO_COPY)  # device residency
    plan = binding.Plan(n, dtype="f64", residency="host", flags=binding.ZERO_COPY)
    s = synth.system(2, n)
    dv = [torch.as_tensor(s[k]).cuda() for k in "abcd"]
    with pytest.raises(binding.TpsError):
        plan.solve_host_async(*dv, torch.empty(n, dtype=torch.float64, device="cuda"))


def test_trace_reports_stage_times():
    n = 1 << 20
    g = synth.system_device(9, n)
    x = torch.empty_like(g["b"])
    plan = binding.Plan(n, dtype="f64_df", m=32, flags=binding.TRACE)
    for _ in range(3):
        plan.solve(g["a"], g["b"], g["c"], g["d"], x)
    info = plan.query()
    s1, s2, s3, tot = info["stage_ms"]
    assert s1 > 0 and s2 > 0 and s3 > 0 and tot >= s1 + s3


@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32"])
def test_unaligned_arrays_take_the_direct_path(dtype):
    """Arrays offset by one element are not 16-byte aligned, so the kernels
    read global memory directly instead of using TMA bulk copies."""
    n = 100003
    s = synth.system(6 + n, n)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    if dtype == "f32":
        s = synth.to_f32(s)
    buf = {k: torch.zeros(n + 1, dtype=tdt, device="cuda") for k in "abcdx"}
    for k in "abcd":
        buf[k][1:] = torch.as_tensor(s[k]).to(tdt).cuda()
    views = [buf[k][1:] for k in "abcdx"]
    assert views[0].data_ptr() % 16 != 0
    plan = binding.Plan(n, dtype=dtype, m=32)
    plan.solve(*views)
    torch.cuda.synchronize()
    assert plan.query()["status"] == 0
    a, b, c, d = (np.asarray(s[k], dtype=np.float64) for k in "abcd")
    ref = oracle.thomas(a, b, c, d)
    tol = F32_FWD if dtype == "f32" else F64_FWD
    assert oracle.rel_forward_error(views[4].cpu().numpy().astype(np.float64), ref) <= tol


def test_graph_mode_replays_and_recaptures():
    n = 300001
    plan = binding.Plan(n, dtype="f64_df", flags=binding.GRAPH | binding.TRACE)
    bufs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(5)]
    for seed in (1, 2):  # same pointers, new data: replay
        s = synth.system(seed, n)
        for t, k in zip(bufs, "abcd"):
            t.copy_(torch.as_tensor(s[k]))
        plan.solve(*bufs)
        torch.cuda.synchronize()
        ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
        assert oracle.rel_forward_error(bufs[4].cpu().numpy(), ref) <= F64_FWD
    info = plan.query()
    assert info["status"] == 0 and info["stage_ms"][3] > 0
    s = synth.system(3, n - 5)  # new n and pointers: recapture
    a, b, c, d = (torch.as_tensor(s[k]).cuda() for k in "abcd")
    x = torch.empty_like(b)
    plan.solve(a, b, c, d, x)
    torch.cuda.synchronize()
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x.cpu().numpy(), ref) <= F64_FWD


@pytest.mark.parametrize("n", [300001, (1 << 21) + 3])
def test_whole_solve_graph_replays_and_recaptures(n):
    """TPS_GRAPH without TRACE: the whole solve (on chip, or level by level
    with an on-chip Stage 2) is one graph; new data in the same buffers is
    solved by the replay, new pointers recapture."""
    plan = binding.Plan(n, dtype="f64_df", flags=binding.GRAPH)
    bufs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(5)]
    for seed in (1, 2):
        s = synth.system(seed, n)
        for t, k in zip(bufs, "abcd"):
            t.copy_(torch.as_tensor(s[k]))
        bufs[4].fill_(float("nan"))
        plan.solve(*bufs)
        torch.cuda.synchronize()
        ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
        assert oracle.rel_forward_error(bufs[4].cpu().numpy(), ref) <= F64_FWD
        assert plan.query()["status"] == 0
    s = synth.system(3, n - 4)
    a, b, c, d = (torch.as_tensor(s[k]).cuda() for k in "abcd")
    x = torch.empty_like(b)
    plan.solve(a, b, c, d, x)
    torch.cuda.synchronize()
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x.cpu().numpy(), ref) <= F64_FWD


def test_graph_mode_batched():
    sizes = [1000, 1, 0, 4097, 300]
    off = synth.offsets_from_sizes(sizes)
    n = int(off[-1])
    s = synth.system(9, n, offsets=off)
    a, b, c, d = (torch.as_tensor(s[k]).cuda() for k in "abcd")
    x = torch.empty_like(b)
    plan = binding.Plan(n, dtype="f64_df", batch_max=8, flags=binding.GRAPH)
    offs = torch.as_tensor(off, device="cuda")
    for _ in range(3):
        x.zero_()
        plan.solve_batched(offs, a, b, c, d, x, host_offsets=off)
        torch.cuda.synchronize()
        ref = oracle.thomas_batched(off, s["a"], s["b"], s["c"], s["d"])
        assert oracle.rel_forward_error(x.cpu().numpy(), ref) <= F64_FWD


def test_distinct_plans_from_two_host_threads():
    # two host threads, each with its own plan and stream, solving at the
    # same time (levels route: no cooperative launch), both against the oracle
    import threading

    n = 300001
    systems = [synth.system(60 + i, n) for i in range(2)]
    refs = [oracle.thomas(s["a"], s["b"], s["c"], s["d"]) for s in systems]
    out, errs = [None, None], []

    def work(i):
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                a, b, c, d = (dev(systems[i][k]) for k in "abcd")
                x = torch.empty_like(b)
                plan = binding.Plan(n, dtype=("f64_df", "f64")[i], m=64 * (i + 1),
                                    flags=binding.NO_ONCHIP | binding.GRAPH * i)
                for _ in range(25):
                    plan.solve(a, b, c, d, x)
            st.synchronize()
            out[i] = (x.cpu().numpy(), plan.query())
        except Exception as e:  # surfaced below
            errs.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errs, errs
    for (x, info), ref, s in zip(out, refs, systems):
        assert info["status"] == 0 and info["onchip"] == 0
        assert oracle.rel_forward_error(x, ref) <= F64_FWD
        assert oracle.rel_residual(s["a"], s["b"], s["c"], s["d"], x) <= F64_RES
