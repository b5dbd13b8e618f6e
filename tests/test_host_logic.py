"""Host-side logic of libtps, no GPU: the paper's stream rule (Eq. 4, 6, 7)
against Table 4, and the host MLP forward pass against the fp64 oracle."""
import ctypes

import numpy as np
import pytest

from oracle import heuristic, mlp
from paper_2501_05938_gb300 import binding
from paper_2501_05938_gb300 import build as tps_build


@pytest.fixture(scope="module")
def lib():
    tps_build.build()
    L = binding.lib()
    L.tps_paper_predict_streams.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_double]
    L.tps_paper_predict_streams.restype = ctypes.c_int32
    L.tps_mlp_forward_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.tps_mlp_forward_host.restype = None
    return L


def test_paper_rule_reproduces_table4(lib, golden):
    for size, n_act, n_pre in golden("table4_opt_streams.txt"):
        assert lib.tps_paper_predict_streams(float(size), None, None, None, 0.0) == int(n_pre)


def test_paper_rule_matches_oracle_with_refit_coefficients(lib):
    rng = np.random.default_rng(0)
    for _ in range(200):
        sm = np.array([rng.uniform(1e-8, 1e-5), rng.uniform(0, 0.5)])
        small = np.array([rng.uniform(0, 1e-6), rng.uniform(0, 1), rng.uniform(-0.2, 0.2)])
        big = np.array([rng.uniform(0, 1e-7), rng.uniform(0, 0.2), rng.uniform(0, 1)])
        size = float(10 ** rng.uniform(3, 8.5))
        got = lib.tps_paper_predict_streams(size, sm.ctypes.data, small.ctypes.data,
                                            big.ctypes.data, 1e6)
        ref = heuristic.predict_streams(size, tuple(sm), tuple(small), tuple(big))
        assert got == ref


def flat(p):
    return np.concatenate([p[k].ravel() for k, _ in mlp.SHAPES]).astype(np.float32)


def test_host_forward_matches_fp64_oracle(lib):
    p = mlp.init_params(3)
    w = flat(p)
    assert w.size == 4675
    rng = np.random.default_rng(1)
    for _ in range(50):
        x = rng.uniform(-2, 2, 4).astype(np.float32)
        y = np.zeros(3, dtype=np.float32)
        lib.tps_mlp_forward_host(w.ctypes.data, x.ctypes.data, y.ctypes.data)
        pf = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
        ref, _ = mlp.forward(pf, x.astype(np.float64)[None, :])
        np.testing.assert_allclose(y, ref[0], rtol=1e-4, atol=1e-5)
