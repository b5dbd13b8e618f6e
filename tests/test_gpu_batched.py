"""Batched uneven solve (packed systems) through the C ABI against the
oracle's per-system Thomas solve.  The entries the convention says are never
read (a on each system's first row, c on its last) are poisoned to prove it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2501_05938_gb300 import binding, synth

pytestmark = pytest.mark.gpu

TOL = {"f64": (1e-10, 1e-12), "f64_df": (1e-10, 1e-12), "f32": (1e-5, 1e-5),
       "mixed": (1e-10, 1e-12)}


def poisoned(s, off):
    a, c = s["a"].copy(), s["c"].copy()
    for i in range(len(off) - 1):
        if off[i + 1] > off[i]:
            a[off[i]] = 1e3
            c[off[i + 1] - 1] = -1e3
    return a, c


def run_batch(dtype, sizes, seed=5, m=0):
    off = synth.offsets_from_sizes(sizes)
    n = int(off[-1])
    s = synth.system(seed, n, offsets=off)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    npdt = np.float32 if dtype == "f32" else np.float64
    a, c = poisoned(s, off)
    b, d = s["b"], s["d"]
    if dtype == "f32":
        a, b, c, d = (v.astype(np.float32) for v in (a, b, c, d))
    dev = [torch.as_tensor(np.ascontiguousarray(v)).to("cuda", tdt) for v in (a, b, c, d)]
    x = torch.empty(n, dtype=tdt, device="cuda")
    offs = torch.as_tensor(off, device="cuda")
    plan = binding.Plan(max(n, 1), dtype=dtype, batch_max=len(sizes), m=m)
    plan.solve_batched(offs, *dev, x, host_offsets=off)
    torch.cuda.synchronize()
    info = plan.query()
    s64 = {k: np.asarray(v, dtype=npdt).astype(np.float64) for k, v in
           zip("abcd", (s["a"], b, s["c"], d))}
    ref = oracle.thomas_batched(off, s64["a"], s64["b"], s64["c"], s64["d"])
    xs = x.cpu().numpy().astype(np.float64)
    return info, xs, ref, s64, off


# mixed: the refinement's corrections run fused into level 0, so its residual
# (formed in Stage 1) must not read the poisoned couplings either
@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32", "mixed"])
@pytest.mark.parametrize("sizes,m", [([1], 32), ([5, 0, 1, 2], 32), ([40, 24], 8),
                                     ([0, 300, 1, 1, 2, 65, 64, 63, 0, 1000], 32),
                                     ([1000, 17, 3000, 1, 4097], 64), ([7] * 300, 16),
                                     ([70000, 1, 129, 65537], 0)])
def test_small_batches(dtype, sizes, m):
    info, xs, ref, s64, off = run_batch(dtype, sizes, m=m)
    assert info["status"] == 0, info
    if dtype == "mixed" and sum(sizes) > 64:
        assert info["refine_fused"]
    fwd, res = TOL[dtype]
    assert oracle.rel_forward_error(xs, ref) <= fwd
    r = oracle.residual_batched(off, s64["a"], s64["b"], s64["c"], s64["d"], xs)
    assert np.max(np.abs(r)) / np.max(np.abs(s64["d"])) <= res


def test_device_offsets_without_host_copy():
    sizes = [100, 200, 1, 300]
    off = synth.offsets_from_sizes(sizes)
    n = int(off[-1])
    s = synth.system(8, n, offsets=off)
    dev = [torch.as_tensor(s[k]).cuda() for k in "abcd"]
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    plan = binding.Plan(n, dtype="f64_df", batch_max=4, m=16)
    plan.solve_batched(torch.as_tensor(off, device="cuda"), *dev, x)
    torch.cuda.synchronize()
    ref = oracle.thomas_batched(off, s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x.cpu().numpy(), ref) <= 1e-10


def test_batch_argument_checks():
    plan = binding.Plan(100, dtype="f64", batch_max=2)
    offs = torch.as_tensor(np.array([0, 50, 100, 100]), device="cuda")
    z = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.TpsError):  # 3 systems > batch_max
        plan.solve_batched(offs, z, z, z, z, torch.zeros_like(z),
                           host_offsets=np.array([0, 50, 100, 100]))
    with pytest.raises(binding.TpsError):  # decreasing offsets
        plan.solve_batched(offs[:3], z, z, z, z, torch.zeros_like(z),
                           host_offsets=np.array([0, 60, 50]))
    with pytest.raises(binding.TpsError):  # offsets the kernels read must be device memory
        plan.solve_batched(torch.as_tensor(np.array([0, 50, 100])), z, z, z, z,
                           torch.zeros_like(z), host_offsets=np.array([0, 50, 100]))


@pytest.mark.slow
@pytest.mark.parametrize("dtype", ["f64_df", "f32"])
def test_full_batch_4096_log_uniform(dtype):
    """4096 systems, n_i = floor(2^U(8,20)) (the uneven-batch workload)."""
    sizes = synth.batch_sizes(1003, 4096, 8, 20)
    off = synth.offsets_from_sizes(sizes)
    n = int(off[-1])
    g = synth.system_device(1003, n, offsets=off)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dev = [g[k].to(tdt) for k in "abcd"]
    x = torch.empty(n, dtype=tdt, device="cuda")
    plan = binding.Plan(n, dtype=dtype, batch_max=4096)
    plan.solve_batched(torch.as_tensor(off, device="cuda"), *dev, x, host_offsets=off)
    torch.cuda.synchronize()
    assert plan.query()["status"] == 0
    h = [v.cpu().numpy().astype(np.float64) for v in dev]
    del g, dev
    ref = oracle.thomas_batched(off, *h)
    fwd, _ = TOL[dtype]
    assert oracle.rel_forward_error(x.cpu().numpy().astype(np.float64), ref) <= fwd
