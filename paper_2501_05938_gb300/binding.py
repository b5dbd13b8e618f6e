"""ctypes binding of libtps (include/tps.h): argument marshalling only.

Every step of the solve runs in the CUDA library; PyTorch supplies device
memory and the current stream.  If ``libtps.so`` is missing this module
raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("TPS_LIB_PATH") or os.path.join(HERE, "libtps.so")

TPS_OK = 0
STATUS = {0: "TPS_OK", 1: "TPS_ERR_INVALID_ARG", 2: "TPS_ERR_UNSUPPORTED", 3: "TPS_ERR_CUDA",
          4: "TPS_ERR_OOM", 5: "TPS_ERR_ZERO_PIVOT", 6: "TPS_ERR_NO_CONVERGENCE",
          7: "TPS_ERR_TIMEOUT", 8: "TPS_ERR_RANGE"}
DTYPES = {"f64": 0, "f32": 1, "mixed": 2, "f64_df": 3}
RESIDENCY = {"device": 0, "host": 1}
TUNE_PREDICT, TUNE_EXHAUSTIVE, TRACE, EXTERNAL_WORKSPACE, GRAPH, ZERO_COPY, NO_ONCHIP = (
    1, 2, 4, 8, 16, 32, 64)
TRUNCATE = 128
HOST_OVERLAP = 256

# every symbol include/tps.h declares
EXPORTS = ("tps_plan", "tps_plan_destroy", "tps_workspace_size", "tps_set_workspace", "tps_solve",
           "tps_solve_batched", "tps_solve_host_async", "tps_solve_host_many_async",
           "tps_plan_query", "tps_status_string", "tps_version", "tps_measure_fp64_rates")


class PlanDesc(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int64), ("batch_max", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("residency", ctypes.c_int32),
                ("m", ctypes.c_int32), ("m_reduced", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("chunk", ctypes.c_int64), ("tol", ctypes.c_double),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("m", ctypes.c_int32), ("m_reduced", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("chunk", ctypes.c_int64), ("last_correction", ctypes.c_double),
                ("stage_ms", ctypes.c_float * 4), ("workspace_bytes", ctypes.c_size_t),
                ("pageable_ok", ctypes.c_int32), ("onchip", ctypes.c_int32),
                ("refine_fused", ctypes.c_int32)]


class TpsError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


_lib = None


def lib():
    """Load libtps.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2501_05938_gb300.build.build() (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.tps_plan.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(P)]
        L.tps_plan_destroy.argtypes = [P]
        L.tps_workspace_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.tps_set_workspace.argtypes = [P, P, ctypes.c_size_t]
        L.tps_solve.argtypes = [P, I64, P, P, P, P, P, P]
        L.tps_solve_batched.argtypes = [P, I64, P, P, P, P, P, P, P, P]
        L.tps_solve_host_async.argtypes = [P, I64, P, P, P, P, P, P]
        PP = ctypes.POINTER(P)
        L.tps_solve_host_many_async.argtypes = [P, I64, I64, PP, PP, PP, PP, PP, P]
        L.tps_plan_query.argtypes = [P, ctypes.POINTER(Info)]
        L.tps_status_string.argtypes = [I32]
        L.tps_status_string.restype = ctypes.c_char_p
        L.tps_version.argtypes = []
        for f in EXPORTS:
            if f not in ("tps_status_string", "tps_version"):
                getattr(L, f).restype = ctypes.c_int
        L.tps_version.restype = ctypes.c_int
        _lib = L
    return _lib


def check(status, what):
    if status != TPS_OK:
        raise TpsError(status, what)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A tps plan (see tps_plan in include/tps.h)."""

    def __init__(self, n_max, dtype="f64", residency="device", m=0, m_reduced=0, streams=0,
                 chunk=0, batch_max=0, tol=0.0, max_iters=0, flags=0):
        self.desc = PlanDesc(n_max=int(n_max), batch_max=int(batch_max), dtype=DTYPES[dtype],
                             residency=RESIDENCY[residency], m=int(m), m_reduced=int(m_reduced),
                             streams=int(streams), max_iters=int(max_iters), chunk=int(chunk),
                             tol=float(tol), flags=int(flags), reserved=0)
        self.dtype = dtype
        self._h = ctypes.c_void_p()
        check(lib().tps_plan(ctypes.byref(self.desc), ctypes.byref(self._h)), "tps_plan")

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().tps_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_size(self):
        v = ctypes.c_size_t()
        check(lib().tps_workspace_size(self._h, ctypes.byref(v)), "tps_workspace_size")
        return v.value

    def set_workspace(self, buf):
        check(lib().tps_set_workspace(self._h, _ptr(buf), buf.numel() * buf.element_size()),
              "tps_set_workspace")

    def _arrays(self, n, *ts):
        """a, b, c, d, x: contiguous tensors of the plan's I/O type (float32
        for "f32", float64 otherwise), n elements each (the library checks
        where they live)."""
        import torch

        want = torch.float32 if self.dtype == "f32" else torch.float64
        for t in ts:
            if t.dtype != want or not t.is_contiguous() or t.numel() != n:
                raise TpsError(1, f"arrays must be contiguous {want} tensors of {n} elements")

    @staticmethod
    def _offsets(offsets, host_offsets):
        import numpy as np
        import torch

        if offsets is not None and (offsets.dtype != torch.int64 or not offsets.is_contiguous()):
            raise TpsError(1, "offsets must be a contiguous int64 tensor")
        if host_offsets is None:
            return None, None
        h = np.ascontiguousarray(host_offsets, dtype=np.int64)
        return h, ctypes.c_void_p(h.ctypes.data)

    def solve(self, a, b, c, d, x, stream=None):
        """Device-resident solve; a..x are CUDA tensors of n elements."""
        n = b.numel()
        self._arrays(n, a, b, c, d, x)
        check(lib().tps_solve(self._h, n, _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x),
                              _stream(stream)), "tps_solve")
        return x

    def solve_batched(self, offsets, a, b, c, d, x, host_offsets=None, stream=None):
        count = offsets.numel() - 1
        self._arrays(b.numel(), a, b, c, d, x)
        keep, hp = self._offsets(offsets, host_offsets)  # keep: alive during the call
        check(lib().tps_solve_batched(self._h, count, _ptr(offsets), hp, _ptr(a), _ptr(b),
                                      _ptr(c), _ptr(d), _ptr(x), _stream(stream)),
              "tps_solve_batched")
        return x

    def solve_host_async(self, a, b, c, d, x, stream=None):
        """a..x are pinned CPU tensors (ZERO_COPY plans: or pageable ones where
        the device reads pageable memory); returns after enqueueing."""
        n = b.numel()
        self._arrays(n, a, b, c, d, x)
        check(lib().tps_solve_host_async(self._h, n, _ptr(a), _ptr(b), _ptr(c), _ptr(d),
                                         _ptr(x), _stream(stream)), "tps_solve_host_async")
        return x

    def solve_host_many(self, systems, xs, stream=None):
        """tps_solve_host_many_async (plans made with HOST_OVERLAP): systems is
        a list of (a, b, c, d) pinned CPU tensors of n elements, xs the list of
        outputs; consecutive systems overlap on the link.  Returns after
        enqueueing."""
        count = len(systems)
        if len(xs) != count:
            raise TpsError(1, "one output per system")
        n = systems[0][1].numel() if count else 0
        for (a, b, c, d), x in zip(systems, xs):
            self._arrays(n, a, b, c, d, x)
        lists = [(ctypes.c_void_p * max(count, 1))(*[t.data_ptr() for t in col])
                 for col in ([s[i] for s in systems] for i in range(4))]
        xl = (ctypes.c_void_p * max(count, 1))(*[t.data_ptr() for t in xs])
        check(lib().tps_solve_host_many_async(self._h, count, n, *lists, xl, _stream(stream)),
              "tps_solve_host_many_async")
        return xs

    def autotune(self, a, b, c, d, x, reps=3, offsets=None, host_offsets=None, stream=None):
        """tps_autotune: time every block size on these arrays and keep the
        fastest in the plan (plans made with TUNE_EXHAUSTIVE cover the whole
        grid); returns (m, ms per solve)."""
        L = lib()
        P = ctypes.c_void_p
        L.tps_autotune.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, P, P, P,
                                   ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_float)]
        L.tps_autotune.restype = ctypes.c_int
        m, ms = ctypes.c_int32(), ctypes.c_float()
        count = 0 if offsets is None else offsets.numel() - 1
        self._arrays(b.numel(), a, b, c, d, x)
        keep, hp = self._offsets(offsets, host_offsets)  # keep: alive during the call
        check(L.tps_autotune(self._h, b.numel(), count, _ptr(offsets), hp, _ptr(a), _ptr(b),
                             _ptr(c), _ptr(d), _ptr(x), _stream(stream), int(reps),
                             ctypes.byref(m), ctypes.byref(ms)), "tps_autotune")
        return m.value, ms.value

    def query(self):
        info = Info()
        check(lib().tps_plan_query(self._h, ctypes.byref(info)), "tps_plan_query")
        return {"status": info.status, "status_name": STATUS.get(info.status, info.status),
                "iterations": info.iterations, "m": info.m, "m_reduced": info.m_reduced,
                "streams": info.streams, "levels": info.levels, "chunk": info.chunk,
                "last_correction": info.last_correction,
                "stage_ms": list(info.stage_ms), "workspace_bytes": info.workspace_bytes,
                "pageable_ok": bool(info.pageable_ok), "onchip": info.onchip,
                "refine_fused": bool(info.refine_fused)}


def measure_fp64_rates():
    """tps_measure_fp64_rates: fp64 (fma, mul, add) thread instructions per
    second of the current device (synchronises it)."""
    L = lib()
    f = L.tps_measure_fp64_rates
    D = ctypes.POINTER(ctypes.c_double)
    f.argtypes = [D, D, D]
    f.restype = ctypes.c_int
    v = [ctypes.c_double() for _ in range(3)]
    check(f(*(ctypes.byref(t) for t in v)), "tps_measure_fp64_rates")
    return tuple(t.value for t in v)


def status_string(s):
    return lib().tps_status_string(int(s)).decode()


def version():
    return lib().tps_version()
