// C ABI of libtps: plans, workspace, the device-resident solve and the
// host-resident streamed pipeline.  Declarations and contracts: include/tps.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "tps_internal.h"
#include "window_kernels.cuh"

namespace tps {

// Streams and events of the host-resident pipeline (Sec. 2.1-2.2: S streams,
// S a power of two up to the 32 hardware queues).
struct HostPipe {
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev_done1;   // per stream: its Stage-1 work is queued
  std::vector<cudaEvent_t> ev_done3;   // per stream: its Stage-3 work is queued
  cudaEvent_t ev_start = nullptr;      // caller's stream reached the solve
  cudaEvent_t ev_red = nullptr;        // Stage 2 done
  cudaEvent_t ev_up = nullptr;         // every upload (and Stage 1) done
  size_t off_dev = 0;                  // device working copies a, b, c, d, x
};

static tps_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return TPS_OK;
  if (e == cudaErrorMemoryAllocation) return TPS_ERR_OOM;
  return TPS_ERR_CUDA;
}

constexpr int kTraceSlots = 256;

// Streams and events of the host pipeline, grown to at least S.
static cudaError_t ensure_streams(HostPipe* H, int S) {
  cudaError_t e = cudaSuccess;
  while ((int)H->streams.size() < S && e == cudaSuccess) {
    cudaStream_t s;
    cudaEvent_t e1, e3;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    H->streams.push_back(s);
    e = cudaEventCreateWithFlags(&e1, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    H->ev_done1.push_back(e1);
    e = cudaEventCreateWithFlags(&e3, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    H->ev_done3.push_back(e3);
  }
  return e;
}
constexpr int32_t kTuneMin = 16, kTuneMax = 1024;  // autotuner block-size grid

static cudaEvent_t* next_trace(tps_plan_s* P) {
  if (!P->trace_ev) return nullptr;
  const int slot = (int)(P->trace_count % P->trace_slots);
  ++P->trace_count;
  return P->trace_ev + 4 * slot;
}

// Defaults when the caller leaves a parameter at 0 and no predictor is asked
// for.  Block size 128: at n = 2^27 within 1.4% of the best block size on
// every GB300 measured (m = 64 is 1.4% faster on some boxes and 2.1% slower
// on others; tps_autotune picks per box); a small system keeps at least ~4
// blocks per SM so the per-lane serial sweeps run in parallel.
static void default_params(const tps_plan_desc& d, int32_t& m, int32_t& mr, int32_t& S) {
  if (m == 0) {
    m = 128;
    while (m > 8 && d.n_max / m < 152 * 32 * 4) m /= 2;
  }
  if (mr == 0) mr = 32;
  if (S == 0) S = (d.residency == TPS_HOST_PINNED) ? 4 : 1;
}

static size_t workspace_for(tps_plan_s* P, size_t* off_levels_out, size_t* off_dev_out) {
  size_t off = 0;
  off = align_up(off + 64);  // status word, refinement maxima, grid-barrier counter
  P->off_dmax = off;         // per-system range codes (zero between solves)
  off = align_up(off + 4 * kCodes * (size_t)std::max<int64_t>(1, P->desc.batch_max));
  P->off_xch = off;          // interface rows of the on-chip solve
  off = align_up(off + onchip_exchange_bytes());
  *off_levels_out = off;
  if (P->desc.flags & TPS_TRUNCATE) {  // windows are solved on their own: no levels
    P->off_rel = off;
    off = align_up(off + truncate_rel_bytes(P->desc.n_max, P->m, P->m_reduced, P->desc.dtype));
    *off_levels_out = off;
    *off_dev_out = off;
    return off;
  }
  std::vector<LevelPlan> lv;
  const size_t eio = elem_bytes_io(P->desc.dtype);
  const size_t ered = elem_bytes_red(P->desc.dtype);
  int64_t nmax = P->desc.n_max;
  size_t end = build_levels(nmax, P->m, P->m_reduced, eio, ered, off, lv);
  if (P->desc.dtype == TPS_MIXED_F32_F64) {
    // residual r and correction delta (fp64)
    P->off_refine = end;
    end = align_up(end + (size_t)nmax * 8);
    end = align_up(end + (size_t)nmax * 8);
  }
  off = end;
  *off_dev_out = off;
  if (P->desc.residency == TPS_HOST_PINNED) {
    for (int i = 0; i < 5; ++i) off = align_up(off + (size_t)nmax * eio);
  }
  return off;
}

}  // namespace tps

using namespace tps;

extern "C" {

int tps_version(void) { return 100; }

const char* tps_status_string(tps_status s) {
  switch (s) {
    case TPS_OK: return "ok";
    case TPS_ERR_INVALID_ARG: return "invalid argument";
    case TPS_ERR_UNSUPPORTED: return "unsupported";
    case TPS_ERR_CUDA: return "CUDA runtime error";
    case TPS_ERR_OOM: return "out of memory";
    case TPS_ERR_ZERO_PIVOT: return "zero or non-finite pivot";
    case TPS_ERR_NO_CONVERGENCE: return "refinement did not converge";
    case TPS_ERR_TIMEOUT: return "device wait timed out";
    case TPS_ERR_RANGE: return "value outside the range of the arithmetic";
  }
  return "unknown status";
}

tps_status tps_plan(const tps_plan_desc* desc, tps_plan_t* out) {
  if (!out) return TPS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc) return TPS_ERR_INVALID_ARG;
  const tps_plan_desc& d = *desc;
  if (d.n_max < 0 || d.batch_max < 0 || d.reserved != 0) return TPS_ERR_INVALID_ARG;
  if (d.dtype < TPS_F64 || d.dtype > TPS_F64_DF) return TPS_ERR_INVALID_ARG;
  if (d.residency != TPS_DEVICE && d.residency != TPS_HOST_PINNED) return TPS_ERR_INVALID_ARG;
  if (d.m != 0 && (d.m < 2 || d.m > (1 << 20))) return TPS_ERR_INVALID_ARG;
  if (!(d.flags & TPS_TRUNCATE) && d.m_reduced != 0 && (d.m_reduced < 4 || d.m_reduced > (1 << 20)))
    return TPS_ERR_INVALID_ARG;
  if (d.streams != 0 && (d.streams < 1 || d.streams > 32)) return TPS_ERR_INVALID_ARG;
  if (d.chunk < 0 || d.max_iters < 0 || d.tol < 0.0) return TPS_ERR_INVALID_ARG;
  if (d.flags & ~(TPS_TUNE_PREDICT | TPS_TUNE_EXHAUSTIVE | TPS_TRACE | TPS_EXTERNAL_WORKSPACE |
                  TPS_GRAPH | TPS_ZERO_COPY | TPS_NO_ONCHIP | TPS_TRUNCATE | TPS_HOST_OVERLAP))
    return TPS_ERR_INVALID_ARG;
  if (d.flags & TPS_HOST_OVERLAP) {
    if (d.residency != TPS_HOST_PINNED) return TPS_ERR_INVALID_ARG;
    if ((d.flags & TPS_EXTERNAL_WORKSPACE) || d.dtype == TPS_MIXED_F32_F64)
      return TPS_ERR_UNSUPPORTED;
  }
  if (d.flags & TPS_TRUNCATE) {
    // windows of m kept rows and m_reduced halo rows (both even, 0 = choose)
    if (d.residency != TPS_DEVICE || d.dtype == TPS_MIXED_F32_F64) return TPS_ERR_UNSUPPORTED;
    if ((d.m % 2) || (d.m_reduced % 2) || d.m_reduced < 0) return TPS_ERR_INVALID_ARG;
    if ((int64_t)d.m + 2 * (int64_t)d.m_reduced > truncate_rows_max() &&
        !(d.m > 0 && truncate_warp_mb(d.m, d.m_reduced) > 0))
      return TPS_ERR_INVALID_ARG;
  }
  if ((d.flags & TPS_ZERO_COPY) && d.residency != TPS_HOST_PINNED) return TPS_ERR_INVALID_ARG;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return TPS_ERR_CUDA;
  }
  tps_plan_s* P = new (std::nothrow) tps_plan_s();
  if (!P) return TPS_ERR_OOM;
  P->desc = d;
  if (d.flags & TPS_HOST_OVERLAP) P->desc.flags |= TPS_NO_ONCHIP;
  P->device = device;
  P->m = d.m;
  P->m_reduced = d.m_reduced;
  P->streams = d.streams;
  P->chunk = d.chunk;
  if ((d.flags & TPS_TUNE_PREDICT) && !(d.flags & TPS_TRUNCATE)) {
    int32_t pm = 0, ps = 0;
    int64_t pc = 0;
    if (tps_predict_params(&d, &pm, &ps, &pc) == 0) {
      if (P->m == 0) P->m = pm;
      if (P->streams == 0) P->streams = ps;
      if (P->chunk == 0) P->chunk = pc;
    }
  }
  if (d.flags & TPS_TRUNCATE) {
    // halo for tol at a dominance factor of 3/4: q^h <= tol (1 - q) / 2
    if (P->m_reduced == 0) {
      const double tol = d.tol > 0.0 ? d.tol : 1e-12, q = 0.75;
      int h = (int)std::ceil(std::log(tol * (1.0 - q) / 2.0) / std::log(q));
      h += h & 1;
      P->m_reduced = std::min(std::max(h, 2), truncate_rows_max() / 4);
    }
    // the one-warp windows: 32 blocks of kWinBlockMax rows per extended
    // window (the fastest measured: the window's fixed costs -- halo,
    // 64-row interface solve, bound -- spread over the most rows)
    if (P->m == 0) P->m = 32 * kWinBlockMax - 2 * P->m_reduced;
    if (P->m < 2) {
      delete P;
      return TPS_ERR_INVALID_ARG;
    }
  }
  default_params(d, P->m, P->m_reduced, P->streams);

  size_t off_levels = 0, off_dev = 0;
  if (d.flags & TPS_TUNE_EXHAUSTIVE) {
    // the autotuner's smallest block size needs the largest workspace
    const int32_t keep = P->m;
    P->m = kTuneMin;
    P->ws_needed = workspace_for(P, &off_levels, &off_dev);
    P->m = keep;
    size_t o2 = 0, d2 = 0;
    const size_t own = workspace_for(P, &o2, &d2);
    if (own > P->ws_needed) {
      P->ws_needed = own;
      off_dev = d2;
    }
  } else {
    P->ws_needed = workspace_for(P, &off_levels, &off_dev);
  }
  P->off_levels = off_levels;

  if (const char* t = std::getenv("TPS_TEST_ONCHIP_TIMEOUT"))
    P->test_barrier_extra = t[0] == '1';
  // test switch: the mixed solve's corrections as three separate passes
  // on every route (to compare them with the fused step)
  if (const char* t = std::getenv("TPS_TEST_UNFUSED_REFINE"))
    P->test_unfused_refine = t[0] == '1';
  if (d.flags & TPS_ZERO_COPY) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccess, dev) == cudaSuccess)
      P->pageable_ok = v != 0;
    cudaGetLastError();
  }
  if (d.residency == TPS_HOST_PINNED) {
    HostPipe* H = new (std::nothrow) HostPipe();
    if (!H) { delete P; return TPS_ERR_OOM; }
    P->pipe = H;
    H->off_dev = off_dev;
    cudaError_t e = cudaEventCreateWithFlags(&H->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H->ev_red, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H->ev_up, cudaEventDisableTiming);
    if (e == cudaSuccess) e = ensure_streams(H, P->streams);
    if (e != cudaSuccess) {
      tps_plan_destroy(P);
      return cuda_status(e);
    }
  }
  if (d.flags & TPS_TRACE) {
    P->trace_slots = kTraceSlots;
    P->trace_ev = new (std::nothrow) cudaEvent_t[4 * kTraceSlots]();
    if (!P->trace_ev) { tps_plan_destroy(P); return TPS_ERR_OOM; }
    for (int i = 0; i < 4 * kTraceSlots; ++i) {
      if (cudaEventCreate(&P->trace_ev[i]) != cudaSuccess) {
        tps_plan_destroy(P);
        return TPS_ERR_CUDA;
      }
    }
  }
  if (!(d.flags & TPS_EXTERNAL_WORKSPACE)) {
    void* ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, P->ws_needed);
    if (e != cudaSuccess) {
      cudaGetLastError();
      tps_plan_destroy(P);
      return TPS_ERR_OOM;
    }
    P->ws = (unsigned char*)ws;
    P->ws_bytes = P->ws_needed;
    P->ws_owned = true;
    P->d_status = (int*)P->ws;
    P->d_scalars = (double*)(P->ws + 8);
    e = cudaMemset(P->ws, 0, P->off_xch);  // header and range codes
    if (e != cudaSuccess) {
      tps_plan_destroy(P);
      return TPS_ERR_CUDA;
    }
  }
  if (d.flags & TPS_HOST_OVERLAP) {
    // the twin: the same plan with the parameters chosen above, fixed
    tps_plan_desc t = P->desc;
    t.flags &= ~(TPS_HOST_OVERLAP | TPS_TUNE_PREDICT | TPS_TUNE_EXHAUSTIVE | TPS_TRACE);
    t.m = P->m;
    t.m_reduced = P->m_reduced;
    t.streams = P->streams;
    t.chunk = P->chunk;
    tps_status ts = tps_plan(&t, &P->twin);
    if (ts != TPS_OK) {
      P->twin = nullptr;
      tps_plan_destroy(P);
      return ts;
    }
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
      e = cudaStreamCreateWithFlags(&P->lane[i], cudaStreamNonBlocking);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&P->lane_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaGetLastError();
      tps_plan_destroy(P);
      return TPS_ERR_CUDA;
    }
  }
  *out = P;
  return TPS_OK;
}

tps_status tps_plan_destroy(tps_plan_t P) {
  if (!P) return TPS_ERR_INVALID_ARG;
  if (P->pipe) {
    HostPipe* H = P->pipe;
    for (auto s : H->streams) cudaStreamDestroy(s);
    for (auto e : H->ev_done1) cudaEventDestroy(e);
    for (auto e : H->ev_done3) cudaEventDestroy(e);
    if (H->ev_start) cudaEventDestroy(H->ev_start);
    if (H->ev_red) cudaEventDestroy(H->ev_red);
    if (H->ev_up) cudaEventDestroy(H->ev_up);
    delete H;
  }
  if (P->trace_ev) {
    for (int i = 0; i < 4 * P->trace_slots; ++i)
      if (P->trace_ev[i]) cudaEventDestroy(P->trace_ev[i]);
    delete[] P->trace_ev;
  }
  if (P->twin) tps_plan_destroy(P->twin);
  for (auto s : P->lane)
    if (s) cudaStreamDestroy(s);
  for (auto e : P->lane_ev)
    if (e) cudaEventDestroy(e);
  if (P->graph) cudaGraphExecDestroy(P->graph);
  if (P->solve_graph) cudaGraphExecDestroy(P->solve_graph);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  if (P->ws_owned && P->ws) cudaFree(P->ws);
  if (P->d_work) cudaFree(P->d_work);
  delete P;
  return TPS_OK;
}

tps_status tps_workspace_size(tps_plan_t P, size_t* bytes) {
  if (!P || !bytes) return TPS_ERR_INVALID_ARG;
  *bytes = P->ws_needed;
  return TPS_OK;
}

tps_status tps_set_workspace(tps_plan_t P, void* dev_ptr, size_t bytes) {
  if (!P || !dev_ptr) return TPS_ERR_INVALID_ARG;
  if (!(P->desc.flags & TPS_EXTERNAL_WORKSPACE)) return TPS_ERR_INVALID_ARG;
  if (bytes < P->ws_needed || ((uintptr_t)dev_ptr % kAlign) != 0) return TPS_ERR_INVALID_ARG;
  if (!on_plan_device(P) || !device_ptr_ok(dev_ptr, kAlign, P->device)) return TPS_ERR_INVALID_ARG;
  P->ws = (unsigned char*)dev_ptr;
  P->ws_bytes = bytes;
  P->ws_owned = false;
  P->d_status = (int*)P->ws;
  P->d_scalars = (double*)(P->ws + 8);
  return cudaMemset(P->ws, 0, P->off_xch) == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}

}  // extern "C"

namespace tps {

// Device pointer check: managed memory, or device memory of `device`,
// aligned to `align` bytes.
bool device_ptr_ok(const void* p, size_t align, int device) {
  if (!p || ((uintptr_t)p % align) != 0) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged ||
         (at.type == cudaMemoryTypeDevice && at.device == device);
}

// The plan's device is the current one.
bool on_plan_device(const tps_plan_s* P) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return dev == P->device;
}

// Host pointer check: pinned host memory, or (pageable_ok: the device has
// coherent access to pageable memory) memory no CUDA allocator owns.
static bool host_ptr_ok(const void* p, size_t align, bool pageable_ok) {
  if (!p || ((uintptr_t)p % align) != 0) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost || (pageable_ok && at.type == cudaMemoryTypeUnregistered);
}

static bool overlaps(const void* x, const void* y, size_t bytes) {
  const uintptr_t a = (uintptr_t)x, b = (uintptr_t)y;
  return a < b + bytes && b < a + bytes;
}

static tps_status check_solve_args(tps_plan_s* P, int64_t n, const void* a, const void* b,
                                   const void* c, const void* d, void* x, bool host) {
  if (!P) return TPS_ERR_INVALID_ARG;
  if (n < 0 || n > P->desc.n_max) return TPS_ERR_INVALID_ARG;
  if (!P->ws) return TPS_ERR_INVALID_ARG;  // external workspace not set
  if (!on_plan_device(P)) return TPS_ERR_INVALID_ARG;
  if (n == 0) return TPS_OK;
  const size_t es = elem_bytes_io(P->desc.dtype);
  const void* in[4] = {a, b, c, d};
  const bool pageable = host && (P->desc.flags & TPS_ZERO_COPY) && P->pageable_ok;
  for (const void* p : in) {
    if (host ? !host_ptr_ok(p, es, pageable) : !device_ptr_ok(p, es, P->device))
      return TPS_ERR_INVALID_ARG;
    if (overlaps(p, x, (size_t)n * es)) return TPS_ERR_INVALID_ARG;
  }
  if (host ? !host_ptr_ok(x, es, pageable) : !device_ptr_ok(x, es, P->device))
    return TPS_ERR_INVALID_ARG;
  return TPS_OK;
}

}  // namespace tps

extern "C" {

tps_status tps_solve(tps_plan_t P, int64_t n, const void* a, const void* b, const void* c,
                     const void* d, void* x, void* stream) {
  tps_status st = check_solve_args(P, n, a, b, c, d, x, false);
  if (st != TPS_OK || n == 0) return st;
  cudaStream_t s = (cudaStream_t)stream;
  P->last_stream = s;
  if (P->desc.flags & TPS_TRUNCATE) return run_truncated(P, n, a, b, c, d, x, s);
  std::vector<LevelPlan> lv;
  build_levels(n, P->m, P->m_reduced, elem_bytes_io(P->desc.dtype),
               elem_bytes_red(P->desc.dtype), P->off_levels, lv);
  P->last_levels = (int32_t)lv.size();
  if (P->desc.dtype == TPS_MIXED_F32_F64)
    return run_refine(P, n, (const double*)a, (const double*)b, (const double*)c,
                      (const double*)d, (double*)x, s, lv, nullptr, 0);
  return run_solve(P, n, a, b, c, d, x, s, lv, next_trace(P));
}

tps_status tps_solve_batched(tps_plan_t P, int64_t count, const int64_t* offsets,
                             const int64_t* host_offsets, const void* a, const void* b,
                             const void* c, const void* d, void* x, void* stream) {
  if (!P || count < 0 || (count > 0 && !offsets)) return TPS_ERR_INVALID_ARG;
  if (count > P->desc.batch_max) return TPS_ERR_INVALID_ARG;
  if (P->desc.flags & TPS_TRUNCATE) return TPS_ERR_UNSUPPORTED;
  if (count == 0) return TPS_OK;
  if (!on_plan_device(P) || !device_ptr_ok(offsets, 8, P->device)) return TPS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t n = 0;
  if (host_offsets) {
    if (host_offsets[0] != 0) return TPS_ERR_INVALID_ARG;
    for (int64_t i = 0; i < count; ++i)
      if (host_offsets[i + 1] < host_offsets[i]) return TPS_ERR_INVALID_ARG;
    n = host_offsets[count];
  } else {
    int64_t ends[2];
    if (cudaMemcpyAsync(ends, offsets + count - 1, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return TPS_ERR_CUDA;
    n = ends[1];
  }
  tps_status st = check_solve_args(P, n, a, b, c, d, x, false);
  if (st != TPS_OK || n == 0) return st;
  P->last_stream = s;
  std::vector<LevelPlan> lv;
  build_levels(n, P->m, P->m_reduced, elem_bytes_io(P->desc.dtype),
               elem_bytes_red(P->desc.dtype), P->off_levels, lv);
  P->last_levels = (int32_t)lv.size();
  // system boundaries strictly inside [0, n): offsets[1 .. count-1]
  const int64_t* bnd = count > 1 ? offsets + 1 : nullptr;
  const int64_t nbnd = count - 1;
  if (!lv.empty()) {
    lv[0].lv.bnd = bnd;
    lv[0].lv.nbnd = nbnd;
  }
  if (P->desc.dtype == TPS_MIXED_F32_F64)
    return run_refine(P, n, (const double*)a, (const double*)b, (const double*)c,
                      (const double*)d, (double*)x, s, lv, bnd, nbnd);
  return run_solve(P, n, a, b, c, d, x, s, lv, next_trace(P), bnd, nbnd);
}

tps_status tps_solve_host_async(tps_plan_t P, int64_t n, const void* a, const void* b,
                                const void* c, const void* d, void* x, void* stream) {
  if (!P) return TPS_ERR_INVALID_ARG;
  if (!P->pipe) return TPS_ERR_INVALID_ARG;  // plan not made for host residency
  tps_status st = check_solve_args(P, n, a, b, c, d, x, true);
  if (st != TPS_OK || n == 0) return st;
  if (P->desc.dtype == TPS_MIXED_F32_F64) return TPS_ERR_UNSUPPORTED;
  HostPipe* H = P->pipe;
  cudaStream_t us = (cudaStream_t)stream;
  const size_t es = elem_bytes_io(P->desc.dtype);
  const size_t span = align_up((size_t)P->desc.n_max * es);
  unsigned char* dev[5];
  for (int i = 0; i < 5; ++i) dev[i] = P->ws + H->off_dev + i * span;
  // TPS_ZERO_COPY: a streaming kernel moves each chunk (SM loads and stores
  // on host memory) instead of the copy engines
  const bool zc = (P->desc.flags & TPS_ZERO_COPY) != 0;
  auto copy = [&](void* dst, const void* src, size_t bytes, cudaMemcpyKind kind,
                  cudaStream_t s) -> cudaError_t {
    return zc ? kernel_copy(dst, src, bytes, s) : cudaMemcpyAsync(dst, src, bytes, kind, s);
  };
  const unsigned char* host[5] = {(const unsigned char*)a, (const unsigned char*)b,
                                  (const unsigned char*)c, (const unsigned char*)d,
                                  (const unsigned char*)x};
  std::vector<LevelPlan> lv;
  build_levels(n, P->m, P->m_reduced, es, elem_bytes_red(P->desc.dtype), P->off_levels, lv);
  P->last_levels = (int32_t)lv.size();
  const int S = P->streams;  // the plan's S (the pipe may hold more streams)
  cudaError_t e = cudaEventRecord(H->ev_start, us);
  for (int i = 0; i < S && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(H->streams[i], H->ev_start, 0);
  if (e != cudaSuccess) return TPS_ERR_CUDA;

  if (lv.empty()) {  // small system: one stream, one chunk
    cudaStream_t s0 = H->streams[0];
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
      e = copy(dev[i], host[i], (size_t)n * es, cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess) e = cudaEventRecord(H->ev_up, s0);
    if (e == cudaSuccess) e = base_solve(P, n, dev[0], dev[1], dev[2], dev[3], dev[4], s0);
    if (e == cudaSuccess) e = dcode_check(P, 1, s0);
    if (e == cudaSuccess)
      e = copy((void*)host[4], dev[4], (size_t)n * es, cudaMemcpyDeviceToHost, s0);
    if (e == cudaSuccess) e = cudaEventRecord(H->ev_done3[0], s0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(us, H->ev_done3[0], 0);
    P->last_stream = us;
    return e == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
  }

  // chunks are runs of whole blocks; chunk j goes to stream j % S
  const Level& L0 = lv[0].lv;
  const int64_t rows_per_chunk = P->chunk > 0 ? P->chunk : (n + S - 1) / S;
  int64_t bpc = rows_per_chunk / L0.m;
  if (bpc < 1) bpc = 1;
  const int64_t nch = (L0.p + bpc - 1) / bpc;
  auto chunk_rows = [&](int64_t j, int64_t& kb, int64_t& ke, int64_t& r0, int64_t& r1) {
    kb = j * bpc;
    ke = kb + bpc < L0.p ? kb + bpc : L0.p;
    r0 = kb * L0.m;
    r1 = (ke == L0.p) ? n : ke * L0.m;
  };
  // Stage 1 per chunk, after its upload
  for (int64_t j = 0; j < nch && e == cudaSuccess; ++j) {
    cudaStream_t s = H->streams[j % S];
    int64_t kb, ke, r0, r1;
    chunk_rows(j, kb, ke, r0, r1);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
      e = copy(dev[i] + r0 * es, host[i] + r0 * es, (size_t)(r1 - r0) * es,
               cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = stage1_range(P, lv[0], kb, ke, dev[0], dev[1], dev[2], dev[3], s);
  }
  // join, Stage 2 on stream 0, fork
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    e = cudaEventRecord(H->ev_done1[i], H->streams[i]);
    if (e == cudaSuccess && i > 0) e = cudaStreamWaitEvent(H->streams[0], H->ev_done1[i], 0);
  }
  if (e == cudaSuccess) e = cudaEventRecord(H->ev_up, H->streams[0]);
  if (e == cudaSuccess) e = dcode_check(P, 1, H->streams[0]);
  if (e == cudaSuccess)
    e = (P->desc.flags & TPS_GRAPH) ? reduced_solve_graph(P, lv, H->streams[0])
                                    : reduced_solve(P, lv, H->streams[0]);
  if (e == cudaSuccess) e = cudaEventRecord(H->ev_red, H->streams[0]);
  for (int i = 1; i < S && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(H->streams[i], H->ev_red, 0);
  // Stage 3 per chunk, then its download
  for (int64_t j = 0; j < nch && e == cudaSuccess; ++j) {
    cudaStream_t s = H->streams[j % S];
    int64_t kb, ke, r0, r1;
    chunk_rows(j, kb, ke, r0, r1);
    e = stage3_range(P, lv[0], kb, ke, dev[0], dev[1], dev[2], dev[3], dev[4], s);
    if (e == cudaSuccess)
      e = copy((void*)(host[4] + r0 * es), dev[4] + r0 * es, (size_t)(r1 - r0) * es,
               cudaMemcpyDeviceToHost, s);
  }
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    e = cudaEventRecord(H->ev_done3[i], H->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(us, H->ev_done3[i], 0);
  }
  P->last_stream = us;
  return e == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}

tps_status tps_solve_host_many_async(tps_plan_t P, int64_t count, int64_t n,
                                     const void* const* a, const void* const* b,
                                     const void* const* c, const void* const* d,
                                     void* const* x, void* stream) {
  if (!P || !P->twin || count < 0) return TPS_ERR_INVALID_ARG;
  if (count > 0 && (!a || !b || !c || !d || !x)) return TPS_ERR_INVALID_ARG;
  if (n < 0 || n > P->desc.n_max || !on_plan_device(P)) return TPS_ERR_INVALID_ARG;
  if (count == 0 || n == 0) return TPS_OK;
  // systems k and k+1 run at the same time: an output may not overlap the
  // other one's output or inputs (each call checks its own arrays)
  const size_t bytes = (size_t)n * elem_bytes_io(P->desc.dtype);
  for (int64_t k = 0; k + 1 < count; ++k) {
    const void* in0[4] = {a[k], b[k], c[k], d[k]};
    const void* in1[4] = {a[k + 1], b[k + 1], c[k + 1], d[k + 1]};
    if (overlaps(x[k], x[k + 1], bytes)) return TPS_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i)
      if (overlaps(x[k], in1[i], bytes) || overlaps(x[k + 1], in0[i], bytes))
        return TPS_ERR_INVALID_ARG;
  }
  tps_plan_s* T = P->twin;  // follows the plan's (possibly autotuned) parameters
  T->m = P->m;
  T->m_reduced = P->m_reduced;
  T->streams = P->streams;
  T->chunk = P->chunk;
  cudaStream_t us = (cudaStream_t)stream;
  cudaError_t e = ensure_streams(T->pipe, T->streams);
  if (e == cudaSuccess) e = cudaEventRecord(P->lane_ev[0], us);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(P->lane[i], P->lane_ev[0], 0);
  if (e != cudaSuccess) return TPS_ERR_CUDA;
  // the uploads of consecutive systems follow one another (system k starts
  // once system k-1's rows are all on the device), so at any time one
  // system uploads while the one before it finishes and downloads, instead
  // of both buffer sets uploading at once and then downloading at once
  tps_status st = TPS_OK;
  for (int64_t k = 0; k < count && st == TPS_OK; ++k) {
    tps_plan_s* Q = (k & 1) ? T : P;
    if (k > 0) {
      tps_plan_s* prev = (k & 1) ? P : T;
      if (cudaStreamWaitEvent(P->lane[k & 1], prev->pipe->ev_up, 0) != cudaSuccess) {
        st = TPS_ERR_CUDA;
        break;
      }
    }
    st = tps_solve_host_async(Q, n, a[k], b[k], c[k], d[k], x[k], P->lane[k & 1]);
  }
  // join both buffer sets back into the caller's stream, also after an error
  // (the systems already enqueued stay ordered before later work)
  e = cudaEventRecord(P->lane_ev[1], P->lane[0]);
  if (e == cudaSuccess) e = cudaEventRecord(P->lane_ev[2], P->lane[1]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(us, P->lane_ev[1], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(us, P->lane_ev[2], 0);
  P->last_stream = us;
  T->last_stream = us;
  if (st != TPS_OK) return st;
  return e == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}

}  // extern "C"

namespace tps {

// Exhaustive search of a host-residency plan: the stream count S over
// {1, 2, 4, 8, 16, 32} and the chunk over {n/S, 2^22, 2^24 rows} on the
// caller's pinned arrays; keeps the fastest (S, chunk) in the plan.
static tps_status autotune_host(tps_plan_s* P, int64_t n, const void* a, const void* b,
                                const void* c, const void* d, void* x, void* stream,
                                int32_t reps, int32_t* best_m, float* best_ms) {
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TPS_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TPS_ERR_CUDA;
  }
  const int32_t keep_S = P->streams;
  const int64_t keep_chunk = P->chunk;
  int32_t bS = keep_S;
  int64_t bc = keep_chunk;
  float best_t = -1.0f;
  tps_status st = TPS_OK;
  if (ensure_streams(P->pipe, 32) != cudaSuccess) st = TPS_ERR_CUDA;
  const int64_t chunks[3] = {0, (int64_t)1 << 22, (int64_t)1 << 24};
  for (int32_t S = 1; S <= 32 && st == TPS_OK; S *= 2) {
    for (int ci = 0; ci < 3 && st == TPS_OK; ++ci) {
      if (chunks[ci] && chunks[ci] * 2 > n) continue;  // fewer than two chunks: same as n/S
      P->streams = S;
      P->chunk = chunks[ci];
      st = tps_solve_host_async(P, n, a, b, c, d, x, stream);  // warm-up
      if (st != TPS_OK) break;
      if (cudaEventRecord(e0, s) != cudaSuccess) { st = TPS_ERR_CUDA; break; }
      for (int r = 0; r < reps && st == TPS_OK; ++r)
        st = tps_solve_host_async(P, n, a, b, c, d, x, stream);
      if (st != TPS_OK) break;
      float ms = 0.0f;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        st = TPS_ERR_CUDA;
        break;
      }
      ms /= reps;
      if (best_t < 0.0f || ms < best_t) {
        best_t = ms;
        bS = S;
        bc = chunks[ci];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const bool ok = st == TPS_OK && best_t >= 0.0f;
  P->streams = ok ? bS : keep_S;
  P->chunk = ok ? bc : keep_chunk;
  if (best_m) *best_m = P->m;
  if (best_ms) *best_ms = best_t;
  return st;
}

}  // namespace tps

extern "C" {

tps_status tps_autotune(tps_plan_t P, int64_t n, int64_t count, const int64_t* offsets,
                        const int64_t* host_offsets, const void* a, const void* b,
                        const void* c, const void* d, void* x, void* stream, int32_t reps,
                        int32_t* best_m, float* best_ms) {
  if (!P || reps < 1 || count < 0) return TPS_ERR_INVALID_ARG;
  if (P->desc.flags & TPS_TRUNCATE) return TPS_ERR_UNSUPPORTED;  // m is the window there
  if (P->pipe)  // host residency: S and chunk instead of m
    return count ? TPS_ERR_INVALID_ARG
                 : autotune_host(P, n, a, b, c, d, x, stream, reps, best_m, best_ms);
  cudaStream_t s = (cudaStream_t)stream;
  auto solve = [&]() -> tps_status {
    return count == 0 ? tps_solve(P, n, a, b, c, d, x, stream)
                      : tps_solve_batched(P, count, offsets, host_offsets, a, b, c, d, x,
                                          stream);
  };
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TPS_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TPS_ERR_CUDA;
  }
  const int32_t keep = P->m;
  int32_t best = keep;
  float best_t = -1.0f;
  tps_status st = TPS_OK;
  for (int32_t m = kTuneMin; m <= kTuneMax && st == TPS_OK; m *= 2) {
    P->m = m;
    size_t o1 = 0, o2 = 0;
    if (workspace_for(P, &o1, &o2) > P->ws_bytes) continue;  // does not fit this plan
    st = solve();  // warm-up
    if (st != TPS_OK) break;
    if (cudaEventRecord(e0, s) != cudaSuccess) { st = TPS_ERR_CUDA; break; }
    for (int r = 0; r < reps && st == TPS_OK; ++r) st = solve();
    if (st != TPS_OK) break;
    float ms = 0.0f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = TPS_ERR_CUDA;
      break;
    }
    ms /= reps;
    if (best_t < 0.0f || ms < best_t) {
      best_t = ms;
      best = m;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->m = (st == TPS_OK && best_t >= 0.0f) ? best : keep;
  if (best_m) *best_m = P->m;
  if (best_ms) *best_ms = best_t;
  return st;
}

tps_status tps_plan_query(tps_plan_t P, tps_info* out) {
  if (!P || !out) return TPS_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->m = P->m;
  out->m_reduced = P->m_reduced;
  out->streams = P->streams;
  out->chunk = P->chunk;
  out->levels = P->last_levels;
  out->iterations = P->last_iters;
  out->last_correction = P->last_corr;
  out->workspace_bytes = P->ws_needed;
  out->pageable_ok = (P->desc.flags & TPS_ZERO_COPY) && P->pageable_ok ? 1 : 0;
  out->onchip = P->last_onchip;
  out->refine_fused = P->last_refine_fused;
  for (int i = 0; i < 4; ++i) out->stage_ms[i] = P->stage_ms[i];
  if (!P->ws) return TPS_OK;
  cudaStream_t s = P->last_stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TPS_ERR_CUDA;
  if (P->trace_ev && P->trace_count > 0) {
    const int64_t cnt = P->trace_count < P->trace_slots ? P->trace_count : P->trace_slots;
    double acc[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < cnt; ++i) {
      cudaEvent_t* ev = P->trace_ev + 4 * i;
      float t;
      if (cudaEventElapsedTime(&t, ev[0], ev[1]) == cudaSuccess) acc[0] += t;
      if (cudaEventElapsedTime(&t, ev[1], ev[2]) == cudaSuccess) acc[1] += t;
      if (cudaEventElapsedTime(&t, ev[2], ev[3]) == cudaSuccess) acc[2] += t;
      if (cudaEventElapsedTime(&t, ev[0], ev[3]) == cudaSuccess) acc[3] += t;
    }
    cudaGetLastError();
    for (int i = 0; i < 4; ++i) P->stage_ms[i] = (float)(acc[i] / cnt);
    for (int i = 0; i < 4; ++i) out->stage_ms[i] = P->stage_ms[i];
    P->trace_count = 0;
  }
  int word = 0;
  if (cudaMemcpy(&word, P->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return TPS_ERR_CUDA;
  if (cudaMemset(P->d_status, 0, sizeof(int)) != cudaSuccess) return TPS_ERR_CUDA;
  if (P->twin && P->twin->ws) {  // the systems the twin solved
    int tw = 0;
    if (cudaStreamSynchronize(P->twin->last_stream) != cudaSuccess ||
        cudaMemcpy(&tw, P->twin->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(P->twin->d_status, 0, sizeof(int)) != cudaSuccess)
      return TPS_ERR_CUDA;
    word |= tw;
  }
  int32_t status = TPS_OK;
  if (word & ST_BAD_PIVOT) status = TPS_ERR_ZERO_PIVOT;
  else if (word & ST_TIMEOUT) status = TPS_ERR_TIMEOUT;
  else if (word & ST_RANGE) status = TPS_ERR_RANGE;
  else if ((word & ST_NO_CONVERGENCE) || P->host_status == TPS_ERR_NO_CONVERGENCE)
    status = TPS_ERR_NO_CONVERGENCE;
  P->host_status = TPS_OK;
  out->status = status;
  if (P->desc.flags & TPS_TRUNCATE) {  // the largest window bound of the last solve
    unsigned bits = 0;
    if (cudaMemcpy(&bits, P->ws + 8, sizeof(bits), cudaMemcpyDeviceToHost) != cudaSuccess)
      return TPS_ERR_CUDA;
    float bound;
    std::memcpy(&bound, &bits, sizeof(bound));
    out->last_correction = bound;
  }
  return TPS_OK;
}

}  // extern "C"
