// Recursive device-resident partition solve: Stage 1 on the input, the same
// method on the reduced interface system (Stage 2) until it fits one warp,
// then Stage 3 back up the levels.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "tps_internal.h"

namespace tps {

Level make_level(int64_t n, int m, int R) {
  Level lv{};
  lv.n = n;
  lv.m = m;
  int64_t p = (n + m - 1) / m;
  int64_t last = n - (p - 1) * (int64_t)m;
  if (last == 1 && p > 1) {  // merge a one-row tail into the previous block
    p -= 1;
    last = m + 1;
  }
  lv.p = p;
  lv.k_begin = 0;
  lv.k_end = p;
  lv.bnd = nullptr;
  lv.nbnd = 0;
  lv.llast = (int32_t)last;
  // checkpoint slots: a block of length L has floor((L - 2) / R) of them;
  // size for the longest block (m + 1) so the count is monotone in n
  lv.ncap = (m + 1 - 2) >= R ? (m + 1 - 2) / R : 0;
  return lv;
}

size_t build_levels(int64_t n, int m0, int mr, size_t top_elem, size_t red_elem, size_t base,
                    std::vector<LevelPlan>& out) {
  out.clear();
  size_t off = base;
  int64_t N = n;
  size_t elem = top_elem;
  int m = m0;
  while (N > kBaseMax) {
    LevelPlan L{};
    L.R = chunk_rows(elem);
    L.lv = make_level(N, m, L.R);
    const int64_t nr = 2 * L.lv.p;
    for (int i = 0; i < 5; ++i) {
      L.off_red[i] = off;
      off = align_up(off + (size_t)nr * red_elem);
    }
    const size_t nck = (size_t)L.lv.ncap * (size_t)L.lv.p;
    for (int i = 0; i < 3; ++i) {
      L.off_ck[i] = off;
      off = align_up(off + nck * red_elem);
    }
    out.push_back(L);
    N = nr;
    elem = red_elem;
    m = mr;
  }
  return off;
}

size_t elem_bytes_io(int dtype) { return dtype == TPS_F32 ? 4 : 8; }
size_t elem_bytes_red(int dtype) {
  return (dtype == TPS_F32 || dtype == TPS_MIXED_F32_F64) ? 4 : 8;
}

// ------------------------------------------------------------------ launchers
// 16-byte copies need 16-byte aligned arrays and blocks that start on a
// 16-byte boundary (m a multiple of the 16-byte vector); otherwise the
// kernels copy element by element.
template <class Tin>
static bool vec16_ok(int m, const void* const* ptrs, int n) {
  constexpr int kVec = 16 / (int)sizeof(Tin);
  if (m % kVec) return false;
  for (int i = 0; i < n; ++i)
    if ((uintptr_t)ptrs[i] % 16) return false;
  return true;
}

template <class K>
static cudaError_t set_smem(K kernel, size_t smem, bool& done) {
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e == cudaSuccess) done = true;
  return e;
}

// Stage 1 streams chunks of K rows (or a multiple) and writes a checkpoint
// every K rows, K being Stage 3's chunk length.
#ifndef TPS_STAGE1_MUL
#define TPS_STAGE1_MUL 1  // Stage-1 chunk rows = K * TPS_STAGE1_MUL (measured best: 1)
#endif
template <class Ar, class Tin, class Tred, int K>
static cudaError_t launch_stage1(const Level& lv, const Tin* a, const Tin* b, const Tin* c,
                                 const Tin* d, Tred* ra, Tred* rb, Tred* rc, Tred* rd, Tred* cg,
                                 Tred* cy, Tred* cv, int* status, cudaStream_t s) {
  constexpr int W = kWarpsPerCta;
  constexpr int R = K * TPS_STAGE1_MUL;
  const size_t smem = Tile<Tin, R>::kBytesPerWarp * W;
  const int64_t warps = (lv.k_end - lv.k_begin + 31) / 32;
  const unsigned grid = (unsigned)((warps + W - 1) / W);
  if (grid == 0) return cudaSuccess;
  const void* ptrs[4] = {a, b, c, d};
  cudaError_t e;
  if (vec16_ok<Tin>(lv.m, ptrs, 4)) {
    static bool done = false;
    auto k = k_stage1<Ar, Tin, Tred, R, K, W, true>;
    if ((e = set_smem(k, smem, done)) != cudaSuccess) return e;
    k<<<grid, 32 * W, smem, s>>>(lv, a, b, c, d, ra, rb, rc, rd, cg, cy, cv, status);
  } else {
    static bool done = false;
    auto k = k_stage1<Ar, Tin, Tred, R, K, W, false>;
    if ((e = set_smem(k, smem, done)) != cudaSuccess) return e;
    k<<<grid, 32 * W, smem, s>>>(lv, a, b, c, d, ra, rb, rc, rd, cg, cy, cv, status);
  }
  return cudaGetLastError();
}

template <class Ar, class Tin, class Tred, int R>
static cudaError_t launch_stage3(const Level& lv, const Tin* a, const Tin* b, const Tin* c,
                                 const Tin* d, const Tred* xr, const Tred* cg, const Tred* cy,
                                 const Tred* cv, Tin* x, int* status, cudaStream_t s) {
  constexpr int W = kWarpsPerCta;
  const size_t smem = Tile3<Tin, Tred, R>::kBytesPerWarp * W;
  const int64_t warps = (lv.k_end - lv.k_begin + 31) / 32;
  const unsigned grid = (unsigned)((warps + W - 1) / W);
  if (grid == 0) return cudaSuccess;
  const void* ptrs[5] = {a, b, c, d, x};
  cudaError_t e;
  if (vec16_ok<Tin>(lv.m, ptrs, 5)) {
    static bool done = false;
    auto k = k_stage3<Ar, Tin, Tred, R, W, true>;
    if ((e = set_smem(k, smem, done)) != cudaSuccess) return e;
    k<<<grid, 32 * W, smem, s>>>(lv, a, b, c, d, xr, cg, cy, cv, x, status);
  } else {
    static bool done = false;
    auto k = k_stage3<Ar, Tin, Tred, R, W, false>;
    if ((e = set_smem(k, smem, done)) != cudaSuccess) return e;
    k<<<grid, 32 * W, smem, s>>>(lv, a, b, c, d, xr, cg, cy, cv, x, status);
  }
  return cudaGetLastError();
}

template <class Ar, class Tin, class Tred>
static cudaError_t run_levels(tps_plan_s* P, const std::vector<LevelPlan>& levels, size_t idx,
                              int64_t n, const Tin* a, const Tin* b, const Tin* c, const Tin* d,
                              Tin* x, cudaStream_t s) {
  if (idx == levels.size()) {
    if (n <= 0) return cudaSuccess;
    k_base<Ar, Tin, Tin><<<1, 32, 0, s>>>(n, a, b, c, d, x, nullptr, 0, P->d_status);
    return cudaGetLastError();
  }
  const LevelPlan& L = levels[idx];
  constexpr int R = kChunkRows<Tin>;
  Tred* red[5];
  for (int i = 0; i < 5; ++i) red[i] = reinterpret_cast<Tred*>(P->ws + L.off_red[i]);
  Tred* ck[3];
  for (int i = 0; i < 3; ++i) ck[i] = reinterpret_cast<Tred*>(P->ws + L.off_ck[i]);
  cudaError_t e = launch_stage1<Ar, Tin, Tred, R>(L.lv, a, b, c, d, red[0], red[1], red[2], red[3],
                                                  ck[0], ck[1], ck[2], P->d_status, s);
  if (e != cudaSuccess) return e;
  e = run_levels<Ar, Tred, Tred>(P, levels, idx + 1, 2 * L.lv.p, red[0], red[1], red[2], red[3],
                                 red[4], s);
  if (e != cudaSuccess) return e;
  return launch_stage3<Ar, Tin, Tred, R>(L.lv, a, b, c, d, red[4], ck[0], ck[1], ck[2], x,
                                         P->d_status, s);
}

// ------------------------------------------------------------------ kernel copies
// Grid-stride copy in 16-byte vectors (both pointers 16-byte aligned) or
// 4-byte words; consecutive threads move consecutive vectors, so every warp
// instruction covers 512 contiguous bytes of both sides.
__global__ void k_copy16(const float4* __restrict__ src, float4* __restrict__ dst, size_t n16,
                         const uint32_t* __restrict__ src_tail, uint32_t* __restrict__ dst_tail,
                         int tail_words) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += stride)
    dst[i] = src[i];
  if (blockIdx.x == 0 && (int)threadIdx.x < tail_words) dst_tail[threadIdx.x] = src_tail[threadIdx.x];
}
__global__ void k_copy4(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, size_t n4) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride)
    dst[i] = src[i];
}

cudaError_t kernel_copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  if ((bytes | (uintptr_t)dst | (uintptr_t)src) % 4) return cudaErrorInvalidValue;
  constexpr int kThreads = 256;
  constexpr size_t kMaxBlocks = 152 * 4;  // four CTAs per SM saturate the host link
  if (((uintptr_t)dst | (uintptr_t)src) % 16 == 0) {
    const size_t n16 = bytes / 16;
    const int tail = (int)((bytes % 16) / 4);
    const size_t blocks = std::max<size_t>(1, std::min(kMaxBlocks, (n16 + kThreads - 1) / kThreads));
    k_copy16<<<(unsigned)blocks, kThreads, 0, s>>>(
        static_cast<const float4*>(src), static_cast<float4*>(dst), n16,
        reinterpret_cast<const uint32_t*>(static_cast<const unsigned char*>(src) + n16 * 16),
        reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(dst) + n16 * 16), tail);
  } else {
    const size_t n4 = bytes / 4;
    const size_t blocks = std::max<size_t>(1, std::min(kMaxBlocks, (n4 + kThreads - 1) / kThreads));
    k_copy4<<<(unsigned)blocks, kThreads, 0, s>>>(static_cast<const uint32_t*>(src),
                                                  static_cast<uint32_t*>(dst), n4);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ dtype dispatch
// Level-0 pieces, used by the device path (with optional stage events) and
// by the chunked host pipeline.
template <class F>
static cudaError_t dispatch(int dtype, F&& f) {
  switch (dtype) {
    case TPS_F64: return f(ArF64{}, (double*)nullptr, (double*)nullptr);
    case TPS_F64_DF: return f(ArDF{}, (double*)nullptr, (float2*)nullptr);
    case TPS_F32: return f(ArF32{}, (float*)nullptr, (float*)nullptr);
    case TPS_MIXED_F32_F64: return f(ArF32{}, (double*)nullptr, (float*)nullptr);
  }
  return cudaErrorInvalidValue;
}

cudaError_t stage1_range(tps_plan_s* P, const LevelPlan& L, int64_t kb, int64_t ke,
                         const void* a, const void* b, const void* c, const void* d,
                         cudaStream_t s) {
  return dispatch(P->desc.dtype, [&](auto ar, auto* tin, auto* tred) -> cudaError_t {
    using Ar = decltype(ar);
    using Tin = std::remove_pointer_t<decltype(tin)>;
    using Tred = std::remove_pointer_t<decltype(tred)>;
    constexpr int R = kChunkRows<Tin>;
    Level lv = L.lv;
    lv.k_begin = kb;
    lv.k_end = ke;
    Tred* red[4];
    for (int i = 0; i < 4; ++i) red[i] = reinterpret_cast<Tred*>(P->ws + L.off_red[i]);
    Tred* ck[3];
    for (int i = 0; i < 3; ++i) ck[i] = reinterpret_cast<Tred*>(P->ws + L.off_ck[i]);
    return launch_stage1<Ar, Tin, Tred, R>(lv, (const Tin*)a, (const Tin*)b, (const Tin*)c,
                                           (const Tin*)d, red[0], red[1], red[2], red[3], ck[0],
                                           ck[1], ck[2], P->d_status, s);
  });
}

cudaError_t stage3_range(tps_plan_s* P, const LevelPlan& L, int64_t kb, int64_t ke,
                         const void* a, const void* b, const void* c, const void* d, void* x,
                         cudaStream_t s) {
  return dispatch(P->desc.dtype, [&](auto ar, auto* tin, auto* tred) -> cudaError_t {
    using Ar = decltype(ar);
    using Tin = std::remove_pointer_t<decltype(tin)>;
    using Tred = std::remove_pointer_t<decltype(tred)>;
    constexpr int R = kChunkRows<Tin>;
    Level lv = L.lv;
    lv.k_begin = kb;
    lv.k_end = ke;
    const Tred* xr = reinterpret_cast<const Tred*>(P->ws + L.off_red[4]);
    const Tred* ck[3];
    for (int i = 0; i < 3; ++i) ck[i] = reinterpret_cast<const Tred*>(P->ws + L.off_ck[i]);
    return launch_stage3<Ar, Tin, Tred, R>(lv, (const Tin*)a, (const Tin*)b, (const Tin*)c,
                                           (const Tin*)d, xr, ck[0], ck[1], ck[2], (Tin*)x,
                                           P->d_status, s);
  });
}

// Stage 2: the recursive solve of level 0's reduced system.
cudaError_t reduced_solve(tps_plan_s* P, const std::vector<LevelPlan>& levels, cudaStream_t s) {
  return dispatch(P->desc.dtype, [&](auto ar, auto* tin, auto* tred) -> cudaError_t {
    using Ar = decltype(ar);
    using Tred = std::remove_pointer_t<decltype(tred)>;
    (void)tin;
    const LevelPlan& L = levels[0];
    Tred* red[5];
    for (int i = 0; i < 5; ++i) red[i] = reinterpret_cast<Tred*>(P->ws + L.off_red[i]);
    return run_levels<Ar, Tred, Tred>(P, levels, 1, 2 * L.lv.p, red[0], red[1], red[2], red[3],
                                      red[4], s);
  });
}

// The one-warp solve of a system of at most kBaseMax rows (bnd: first rows
// of packed systems 1.., or null).
cudaError_t base_solve(tps_plan_s* P, int64_t n, const void* a, const void* b, const void* c,
                       const void* d, void* x, cudaStream_t s, const int64_t* bnd,
                       int64_t nbnd) {
  return dispatch(P->desc.dtype, [&](auto ar, auto* tin, auto* tred) -> cudaError_t {
    using Ar = decltype(ar);
    using Tin = std::remove_pointer_t<decltype(tin)>;
    (void)tred;
    k_base<Ar, Tin, Tin><<<1, 32, 0, s>>>(n, (const Tin*)a, (const Tin*)b, (const Tin*)c,
                                          (const Tin*)d, (Tin*)x, bnd, nbnd, P->d_status);
    return cudaGetLastError();
  });
}

// TPS_GRAPH: Stage 2 (every level below the top, many small launches)
// touches only workspace buffers, so one captured graph serves every solve
// with the same level geometry; it is replayed as a single launch.
cudaError_t reduced_solve_graph(tps_plan_s* P, const std::vector<LevelPlan>& levels,
                                cudaStream_t s) {
  const Level& L0 = levels[0].lv;
  const int64_t key[12] = {2 * L0.p, (int64_t)levels.size(), P->m_reduced, (int64_t)P->ws,
                           P->desc.dtype, (int64_t)levels[0].off_red[0], 0, 0, 0, 0, 0, 0};
  bool same = P->graph != nullptr;
  for (int i = 0; i < 12 && same; ++i) same = P->gkey[i] == key[i];
  if (!same) {
    if (P->graph) {
      cudaGraphExecDestroy(P->graph);
      P->graph = nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!P->cap_stream) e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t ec = reduced_solve(P, levels, P->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(P->cap_stream, &g);
    if (ec != cudaSuccess || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return ec != cudaSuccess ? ec : (e != cudaSuccess ? e : cudaErrorUnknown);
    }
    e = cudaGraphInstantiate(&P->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      P->graph = nullptr;
      return e;
    }
    for (int i = 0; i < 12; ++i) P->gkey[i] = key[i];
  }
  return cudaGraphLaunch(P->graph, s);
}

tps_status run_solve(tps_plan_s* P, int64_t n, const void* a, const void* b, const void* c,
                     const void* d, void* x, cudaStream_t s, const std::vector<LevelPlan>& lv,
                     cudaEvent_t* ev, const int64_t* bnd, int64_t nbnd) {
  cudaError_t e = cudaSuccess;
  if (ev) e = cudaEventRecord(ev[0], s);
  if (lv.empty()) {
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = base_solve(P, n, a, b, c, d, x, s, bnd, nbnd);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
  } else {
    if (e == cudaSuccess) e = stage1_range(P, lv[0], 0, lv[0].lv.p, a, b, c, d, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess)
      e = (P->desc.flags & TPS_GRAPH) ? reduced_solve_graph(P, lv, s) : reduced_solve(P, lv, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
    if (e == cudaSuccess) e = stage3_range(P, lv[0], 0, lv[0].lv.p, a, b, c, d, x, s);
  }
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], s);
  return e == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}

}  // namespace tps
