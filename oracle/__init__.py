"""CPU oracle for the tridiagonal partition method -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  The product path (the CUDA
library ``libtps`` and its Python binding) never imports, links or calls it,
and the two share no code.

Contents
  * ``liboracle.so`` (``oracle.c``): serial fp64 Thomas, a serial partition
    solver that follows the method's three stages (Sec. 1, Sec. 2.2), the
    same with Stages 1 and 3 over host threads (the multi-core CPU
    baseline), dense Gaussian elimination with partial pivoting, residuals
    and norms.
  * ``heuristic.py``: the paper's stream-count time models (Eq. 1-7) and the
    optimum-stream rule (Eq. 6), in plain Python.
  * ``mlp.py``: the launch-parameter MLP forward/backward in fp64 numpy.
  * ``refine.py``: mixed-precision iterative refinement, step by step.
  * ``truncated.py``: truncated decoupling (windows with halos) and its
    per-window error bound.

Every function takes and returns numpy arrays; the C routines run on the
host in plain fp64 (compiled with ``-ffp-contract=off``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ORC_OK, ORC_ZERO_PIVOT, ORC_BAD_ARG, ORC_NO_MEMORY = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (plain gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-pthread", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int64
        lib.orc_thomas.argtypes = [I, P, P, P, P, P]
        lib.orc_thomas_batched.argtypes = [I, P, P, P, P, P, P]
        lib.orc_partition.argtypes = [I, I, P, P, P, P, P]
        lib.orc_partition_ex.argtypes = [I, I, P, P, P, P, P, P, P, P, P]
        lib.orc_partition_threaded.argtypes = [I, I, P, P, P, P, P, ctypes.c_int]
        lib.orc_partition_reduced_size.argtypes = [I, I]
        lib.orc_partition_reduced_size.restype = I
        lib.orc_dense_ge.argtypes = [I, P, P, P, P, P]
        lib.orc_thomas_f32.argtypes = [I, P, P, P, P, P]
        lib.orc_residual.argtypes = [I, P, P, P, P, P, P]
        lib.orc_residual.restype = None
        lib.orc_maxabs_diff.argtypes = [I, P, P, P, P]
        lib.orc_maxabs_diff.restype = None
        for f in ("orc_thomas", "orc_thomas_batched", "orc_partition", "orc_partition_ex",
                  "orc_partition_threaded", "orc_dense_ge", "orc_thomas_f32"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _f64(v):
    return np.ascontiguousarray(v, dtype=np.float64)


def _p(v):
    return v.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != ORC_OK:
        raise OracleError(f"{what}: status {st}")


def thomas(a, b, c, d):
    """Serial fp64 Thomas solve of one tridiagonal system (a[0], c[-1] unused)."""
    a, b, c, d = map(_f64, (a, b, c, d))
    n = b.shape[0]
    x = np.empty(n, dtype=np.float64)
    _check(_load().orc_thomas(n, _p(a), _p(b), _p(c), _p(d), _p(x)), "thomas")
    return x


def thomas_f32(a, b, c, d):
    """Thomas carried out in IEEE binary32 arithmetic (inputs rounded to f32)."""
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float32) for v in (a, b, c, d))
    n = b.shape[0]
    x = np.empty(n, dtype=np.float32)
    _check(_load().orc_thomas_f32(n, _p(a), _p(b), _p(c), _p(d), _p(x)), "thomas_f32")
    return x


def thomas_batched(offsets, a, b, c, d):
    """Thomas on each packed system ``offsets[s] .. offsets[s+1]-1``."""
    a, b, c, d = map(_f64, (a, b, c, d))
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    x = np.empty(b.shape[0], dtype=np.float64)
    _check(_load().orc_thomas_batched(off.shape[0] - 1, _p(off), _p(a), _p(b), _p(c), _p(d),
                                      _p(x)), "thomas_batched")
    return x


def partition(a, b, c, d, m, return_reduced=False):
    """Serial partition-method solve with blocks of ``m`` rows.

    With ``return_reduced`` also returns the reduced interface system
    (ra, rb, rc, rd) in the unknown order f_0, l_0, f_1, l_1, ...
    """
    a, b, c, d = map(_f64, (a, b, c, d))
    n = b.shape[0]
    lib = _load()
    x = np.empty(n, dtype=np.float64)
    if not return_reduced:
        _check(lib.orc_partition(n, int(m), _p(a), _p(b), _p(c), _p(d), _p(x)), "partition")
        return x
    nr = lib.orc_partition_reduced_size(n, int(m))
    red = [np.zeros(max(nr, 1), dtype=np.float64) for _ in range(4)]
    _check(lib.orc_partition_ex(n, int(m), _p(a), _p(b), _p(c), _p(d), _p(x),
                                *[_p(r) for r in red]), "partition")
    return x, tuple(r[:nr] for r in red)


def partition_threaded(a, b, c, d, m, threads=None):
    """The partition solve with Stages 1 and 3 over ``threads`` host threads
    (default: every core of the host), Stage 2 serial: the multi-core CPU
    baseline.  Bit-identical to :func:`partition`."""
    a, b, c, d = map(_f64, (a, b, c, d))
    n = b.shape[0]
    t = int(threads or os.cpu_count() or 1)
    x = np.empty(n, dtype=np.float64)
    _check(_load().orc_partition_threaded(n, int(m), _p(a), _p(b), _p(c), _p(d), _p(x), t),
           "partition_threaded")
    return x


def reduced_size(n, m):
    return int(_load().orc_partition_reduced_size(int(n), int(m)))


def dense_ge(a, b, c, d):
    """Dense Gaussian elimination with partial pivoting (n <= 512)."""
    a, b, c, d = map(_f64, (a, b, c, d))
    n = b.shape[0]
    x = np.empty(n, dtype=np.float64)
    _check(_load().orc_dense_ge(n, _p(a), _p(b), _p(c), _p(d), _p(x)), "dense_ge")
    return x


def residual(a, b, c, d, x):
    """r = d - A x in fp64 (a[0], c[-1] unused)."""
    a, b, c, d, x = map(_f64, (a, b, c, d, x))
    r = np.empty(b.shape[0], dtype=np.float64)
    _load().orc_residual(b.shape[0], _p(a), _p(b), _p(c), _p(d), _p(x), _p(r))
    return r


def residual_batched(offsets, a, b, c, d, x):
    """Residual of packed independent systems (no coupling across systems)."""
    a, b, c, d, x = map(_f64, (a, b, c, d, x))
    r = np.empty(b.shape[0], dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    for s in range(off.shape[0] - 1):
        lo, hi = int(off[s]), int(off[s + 1])
        r[lo:hi] = residual(a[lo:hi], b[lo:hi], c[lo:hi], d[lo:hi], x[lo:hi])
    return r


def rel_forward_error(x, x_ref):
    """||x - x_ref||_inf / ||x_ref||_inf (NaN anywhere counts as infinite)."""
    x, x_ref = _f64(x), _f64(x_ref)
    md, mr = ctypes.c_double(), ctypes.c_double()
    _load().orc_maxabs_diff(x.shape[0], _p(x), _p(x_ref), ctypes.byref(md), ctypes.byref(mr))
    if mr.value == 0.0:
        return md.value
    return md.value / mr.value


def rel_residual(a, b, c, d, x):
    """||d - A x||_inf / ||d||_inf computed in fp64 on the host."""
    r = residual(a, b, c, d, x)
    dn = float(np.max(np.abs(_f64(d)))) if d.shape[0] else 0.0
    rn = float(np.max(np.abs(r))) if r.shape[0] else 0.0
    if not np.isfinite(rn):
        return float("inf")
    return rn / dn if dn > 0 else rn


def normwise_backward_error(a, b, c, d, x):
    """||r|| / (||A|| ||x|| + ||d||) in the infinity norm."""
    a, b, c, d, x = map(_f64, (a, b, c, d, x))
    n = b.shape[0]
    if n == 0:
        return 0.0
    r = residual(a, b, c, d, x)
    rows = np.abs(b).copy()
    rows[1:] += np.abs(a[1:])
    rows[:-1] += np.abs(c[:-1])
    return float(np.max(np.abs(r)) / (np.max(rows) * np.max(np.abs(x)) + np.max(np.abs(d))))
