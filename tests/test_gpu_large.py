"""The largest systems: n = 2^31 + 5 rows (17 GB per fp64 array), past the
32-bit element-index range, through the level-by-level route (Stage 2
finishing on chip).  Too large for the serial oracle at test speed, so the
checks are properties that hold at any size: the manufactured solution
x_true (d = A x_true) and the residual d - A x over every row on the device,
plus a sample of rows whose residual is recomputed in fp64 on the host."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_05938_gb300 import binding, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = (1 << 31) + 5
CHUNK = 1 << 28


def free_bytes():
    return torch.cuda.mem_get_info()[0] if torch.cuda.is_available() else 0


@pytest.mark.skipif(torch.cuda.is_available() and free_bytes() < (150 << 30),
                    reason="needs about 150 GB of free device memory")
@pytest.mark.parametrize("dtype", ["f64_df"])
def test_past_the_32_bit_index_range(dtype):
    g = synth.system_device(2031, N)
    x = torch.empty_like(g["b"])
    plan = binding.Plan(N, dtype=dtype, flags=binding.GRAPH)
    plan.solve(g["a"], g["b"], g["c"], g["d"], x)
    torch.cuda.synchronize()
    info = plan.query()
    assert info["status"] == 0 and info["onchip"] == 2, info
    a, b, c, d, xt = g["a"], g["b"], g["c"], g["d"], g["x_true"]
    err = res = 0.0
    xmax = dmax = 0.0
    for lo in range(0, N, CHUNK):
        hi = min(lo + CHUNK, N)
        err = max(err, (x[lo:hi] - xt[lo:hi]).abs().max().item())
        xmax = max(xmax, xt[lo:hi].abs().max().item())
        dmax = max(dmax, d[lo:hi].abs().max().item())
        r = d[lo:hi] - b[lo:hi] * x[lo:hi]
        if lo > 0:
            r -= a[lo:hi] * x[lo - 1:hi - 1]
        else:
            r[1:] -= a[1:hi] * x[0:hi - 1]
        if hi < N:
            r -= c[lo:hi] * x[lo + 1:hi + 1]
        else:
            r[:-1] -= c[lo:hi - 1] * x[lo + 1:hi]
        res = max(res, r.abs().max().item())
        del r
    assert err / xmax <= 1e-10, err / xmax
    assert res / dmax <= 1e-12, res / dmax
    # rows sampled across the whole range (both ends included), residual in fp64 on the host
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[1, N - 2], rng.integers(1, N - 1, 1 << 20)]))
    it = torch.as_tensor(idx, device="cuda")
    av, bv, cv, dv = (t[it].cpu().numpy() for t in (a, b, c, d))
    xm, x0, xp = (x[it + o].cpu().numpy() for o in (-1, 0, 1))
    rs = dv - (av * xm + bv * x0 + cv * xp)
    assert np.max(np.abs(rs)) / dmax <= 1e-12
