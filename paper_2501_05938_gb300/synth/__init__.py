"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

This module only synthesises inputs; it holds none of the solver's
arithmetic.  The numpy functions here and the CUDA kernel in ``synth.cu``
implement the same definition and produce bit-identical arrays.

Random numbers
  SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): a generator seeded with s returns, on its k-th
  call (k >= 1), mix64(s + k * G) with G = 0x9E3779B97F4A7C15 and
      mix64(z): z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
                z = (z ^ (z >> 27)) * 0x94D049BB133111EB
                return z ^ (z >> 31)            (all arithmetic mod 2^64).
  Stream ``st`` of run ``seed`` is the generator seeded with
  key = mix64(seed + st * G); its element i is its (i+1)-th output, so any
  element can be computed on its own.  Uniforms are u = (out >> 11) * 2^-53.

Systems  (a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i])
  streams: 1 -> a, 2 -> b, 3 -> c, 4 -> x_true, 5 -> system sizes
  a = 2u - 1 and c = 2u - 1, with a = 0 on each system's first row and
  c = 0 on its last row;
  kind "paper" (strictly diagonally dominant by at least 1):
      b = (|a| + |c|) + (1 + u)
  kind "ratio" with dominance ratio r > 1:
      b = r * max(|a| + |c|, 2^-20)
  x_true = 2u - 1
  d = (ta + b x_true[i]) + tc, ta = a x_true[i-1] (0 on a first row),
      tc = c x_true[i+1] (0 on a last row), each operation rounded once.
Batched sizes: n_s = floor(2^(lo + (hi - lo) u_s)) from stream 5.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
TWO_M53 = 2.0 ** -53

STREAM_A, STREAM_B, STREAM_C, STREAM_X, STREAM_SIZES = 1, 2, 3, 4, 5
KIND_PAPER, KIND_RATIO = 0, 1
RATIO_FLOOR = 2.0 ** -20


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        s = s + np.uint64(stream) * GOLDEN
    return mix64(s)[0]


def raw(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Outputs start+1 .. start+count of stream ``stream`` (uint64)."""
    key = stream_key(seed, stream)
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key + idx * GOLDEN)


def uniform(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    return (raw(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) * TWO_M53


def _boundaries(n: int, offsets):
    first = np.zeros(n, dtype=bool)
    last = np.zeros(n, dtype=bool)
    if n == 0:
        return first, last
    off = np.asarray(offsets, dtype=np.int64)
    starts = off[:-1][off[1:] > off[:-1]]
    ends = off[1:][off[1:] > off[:-1]] - 1
    first[starts] = True
    last[ends] = True
    return first, last


def system(seed: int, n: int, kind: int = KIND_PAPER, ratio: float = 2.0, offsets=None):
    """Returns dict(a, b, c, d, x_true) of fp64 arrays of length n.

    ``offsets`` (count+1 entries, offsets[0] = 0, offsets[-1] = n) packs
    independent systems back to back; None means one system.
    """
    if offsets is None:
        offsets = np.array([0, n], dtype=np.int64)
    first, last = _boundaries(n, offsets)
    a = 2.0 * uniform(seed, STREAM_A, 0, n) - 1.0
    c = 2.0 * uniform(seed, STREAM_C, 0, n) - 1.0
    a[first] = 0.0
    c[last] = 0.0
    if kind == KIND_PAPER:
        b = (np.abs(a) + np.abs(c)) + (1.0 + uniform(seed, STREAM_B, 0, n))
    elif kind == KIND_RATIO:
        b = ratio * np.maximum(np.abs(a) + np.abs(c), RATIO_FLOOR)
    else:
        raise ValueError("unknown kind")
    x = 2.0 * uniform(seed, STREAM_X, 0, n) - 1.0
    ta = np.zeros(n)
    tc = np.zeros(n)
    if n > 1:
        ta[1:] = a[1:] * x[:-1]
        tc[:-1] = c[:-1] * x[1:]
    ta[first] = 0.0
    tc[last] = 0.0
    d = (ta + b * x) + tc
    return {"a": a, "b": b, "c": c, "d": d, "x_true": x}


def batch_sizes(seed: int, count: int, lo_exp: float, hi_exp: float) -> np.ndarray:
    """n_s = floor(2^(lo + (hi - lo) u_s)) for s = 0 .. count-1."""
    u = uniform(seed, STREAM_SIZES, 0, count)
    return np.floor(np.exp2(lo_exp + (hi_exp - lo_exp) * u)).astype(np.int64)


def offsets_from_sizes(sizes) -> np.ndarray:
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(sizes.shape[0] + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def to_f32(sys_: dict) -> dict:
    """The same system rounded to binary32 (d rounded too, not recomputed)."""
    return {k: np.asarray(v, dtype=np.float32) for k, v in sys_.items()}


# ---------------------------------------------------------------------------
# Device generator (synth.cu, built into libtpssynth.so): same arrays, made
# on the GPU for the sizes the host would take too long on.
# ---------------------------------------------------------------------------
_dev_lib = None


def _device_lib():
    global _dev_lib
    if _dev_lib is None:
        import ctypes
        import os

        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtpssynth.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_2501_05938_gb300.build.build()")
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.tps_synth_system.argtypes = [ctypes.c_uint64, ctypes.c_int64, P, ctypes.c_int64,
                                       ctypes.c_int, ctypes.c_double, P, P, P, P, P, P]
        L.tps_synth_system.restype = ctypes.c_int
        _dev_lib = L
    return _dev_lib


def system_device(seed: int, n: int, kind: int = KIND_PAPER, ratio: float = 2.0, offsets=None,
                  device="cuda", stream=None):
    """Like ``system`` but returns CUDA tensors made on the device.

    ``offsets``: None, or an int64 tensor/array of count+1 entries."""
    import ctypes

    import torch

    out = {k: torch.empty(n, dtype=torch.float64, device=device)
           for k in ("a", "b", "c", "d", "x_true")}
    off_t = None
    count = 1
    if offsets is not None:
        off_t = torch.as_tensor(np.asarray(offsets, dtype=np.int64), device=device)
        count = off_t.numel() - 1
    if stream is None:
        stream = torch.cuda.current_stream()
    st = _device_lib().tps_synth_system(
        ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), n,
        ctypes.c_void_p(off_t.data_ptr()) if off_t is not None else None, count, kind,
        float(ratio), *[ctypes.c_void_p(out[k].data_ptr()) for k in ("a", "b", "c", "d", "x_true")],
        ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        raise RuntimeError(f"tps_synth_system failed with {st}")
    return out
