"""The predictor network's CUDA kernels (forward, loss/backward, Adam)
against the fp64 oracle network, and the host forward pass against the
device one; the exhaustive-search autotuner."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import mlp
from paper_2501_05938_gb300 import binding, synth, tune

pytestmark = pytest.mark.gpu


def flat(p):
    return np.concatenate([p[k].ravel() for k, _ in mlp.SHAPES]).astype(np.float32)


def unflat(w):
    out, o = {}, 0
    for k, shp in mlp.SHAPES:
        n = int(np.prod(shp))
        out[k] = w[o:o + n].reshape(shp).astype(np.float64)
        o += n
    return out


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def setup(B=37, seed=0):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    for k in p:  # non-zero biases so every term is exercised
        if k.startswith("b"):
            p[k] = rng.uniform(-0.1, 0.1, p[k].shape)
    w = flat(p)
    X = rng.uniform(-1, 1, (B, 4)).astype(np.float32)
    T = rng.uniform(-1, 1, (B, 3)).astype(np.float32)
    return w, X, T


def test_forward_matches_host_bitwise_and_oracle():
    L = tune._mlp_lib()
    L.tps_mlp_forward_host.argtypes = [ctypes.c_void_p] * 3
    L.tps_mlp_forward_host.restype = None
    w, X, _ = setup()
    B = X.shape[0]
    dw, dx = torch.as_tensor(w).cuda(), torch.as_tensor(X).cuda()
    y = torch.empty(B, 3, dtype=torch.float32, device="cuda")
    work = torch.empty(int(L.tps_mlp_workspace_floats(B)), dtype=torch.float32, device="cuda")
    assert L.tps_mlp_forward(ptr(dw), B, ptr(dx), ptr(y), ptr(work), None) == 0
    torch.cuda.synchronize()
    yg = y.cpu().numpy()
    for b in range(B):
        yh = np.zeros(3, dtype=np.float32)
        L.tps_mlp_forward_host(w.ctypes.data, X[b].ctypes.data, yh.ctypes.data)
        np.testing.assert_array_equal(yg[b], yh)
    ref, _ = mlp.forward(unflat(w), X.astype(np.float64))
    np.testing.assert_allclose(yg, ref, rtol=1e-4, atol=1e-5)


def test_gradients_match_the_oracle():
    L = tune._mlp_lib()
    w, X, T = setup(B=53, seed=1)
    B = X.shape[0]
    dw, dx, dt = (torch.as_tensor(v).cuda() for v in (w, X, T))
    g = torch.empty_like(dw)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = torch.empty(int(L.tps_mlp_workspace_floats(B)), dtype=torch.float32, device="cuda")
    assert L.tps_mlp_loss_backward(ptr(dw), B, ptr(dx), ptr(dt), ptr(g), ptr(loss), ptr(work),
                                   None) == 0
    torch.cuda.synchronize()
    Lref, gref = mlp.backward(unflat(w), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss.item() - Lref) <= 1e-4 * abs(Lref)
    gg = unflat(g.cpu().numpy())
    for k in gref:
        scale = max(np.max(np.abs(gref[k])), 1e-6)
        assert np.max(np.abs(gg[k] - gref[k])) <= 1e-3 * scale, k


def test_adam_step_matches_the_oracle():
    L = tune._mlp_lib()
    rng = np.random.default_rng(2)
    w = rng.uniform(-1, 1, 4675).astype(np.float32)
    state = {}
    pw = {"w": w.astype(np.float64)}
    dw = torch.as_tensor(w).cuda()
    m = torch.zeros_like(dw)
    v = torch.zeros_like(dw)
    for t in range(1, 4):
        gr = rng.uniform(-1, 1, 4675).astype(np.float32)
        assert L.tps_mlp_adam_step(ptr(dw), ptr(torch.as_tensor(gr).cuda()), ptr(m), ptr(v), t,
                                   1e-2, 0.9, 0.999, 1e-8, None) == 0
        mlp.adam_step(pw, {"w": gr.astype(np.float64)}, state, t, lr=1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(dw.cpu().numpy(), pw["w"], rtol=1e-5, atol=1e-6)


def test_training_on_gpu_reduces_the_loss(tmp_path):
    rng = np.random.default_rng(3)
    rows = []
    for n in [2 ** k for k in range(10, 29, 2)]:
        for m in tune.M_GRID:
            rows.append(dict(kind="device", n=n, batch=1, dtype=0, residency=0, m=m, S=1,
                             chunk=0, ms=1.0 + abs(np.log2(m) - np.log2(n) / 4) + rng.uniform(0, .01),
                             s13_ms=0.0))
    hist = tune.train(rows, str(tmp_path / "w.bin"), steps=1500, log=lambda *_: None)
    assert hist[-1][1] < 0.2 * hist[0][1]
    L = binding.lib()
    L.tps_predict_load.argtypes = [ctypes.c_char_p]
    assert L.tps_predict_load(str(tmp_path / "w.bin").encode()) == 0


def test_autotune_picks_a_block_size_and_stays_correct():
    n = 1 << 20
    s = synth.system(77, n)
    a, b, c, d = (torch.as_tensor(s[k]).cuda() for k in "abcd")
    x = torch.empty_like(b)
    plan = binding.Plan(n, dtype="f64_df", flags=binding.TUNE_EXHAUSTIVE)
    L = binding.lib()
    P = ctypes.c_void_p
    L.tps_autotune.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, P, P, P,
                               ctypes.c_int32, P, P]
    L.tps_autotune.restype = ctypes.c_int
    best = ctypes.c_int32()
    ms = ctypes.c_float()
    st = torch.cuda.current_stream()
    assert L.tps_autotune(plan.handle, n, 0, None, None, ptr(a), ptr(b), ptr(c), ptr(d), ptr(x),
                          P(st.cuda_stream), 2, ctypes.byref(best), ctypes.byref(ms)) == 0
    assert best.value in tune.M_GRID[1:] and ms.value > 0
    assert plan.query()["m"] == best.value
    plan.solve(a, b, c, d, x)
    torch.cuda.synchronize()
    ref = oracle.thomas(s["a"], s["b"], s["c"], s["d"])
    assert oracle.rel_forward_error(x.cpu().numpy(), ref) <= 1e-10
