// Recursive device-resident partition solve: Stage 1 on the input, the same
// method on the reduced interface system (Stage 2) until it fits one warp
// or the GPU's shared memory (the single-launch on-chip solve), then Stage 3
// back up the levels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>
#include <vector>

#include "onchip.cuh"
#include "tps_internal.h"
#include "window_kernels.cuh"

namespace tps {

size_t onchip_exchange_bytes() { return (size_t)4 * 2 * kOcMaxCtas * 8; }
int truncate_rows_max() { return kWinRowsMax; }
int truncate_warp_mb(int R, int h) {
  const int64_t e = (int64_t)R + 2 * (int64_t)h;
  if (R < 2 || h < 0 || e % 32) return 0;
  const int mb = (int)(e / 32);
  return (mb >= kWinBlockMin && mb <= kWinBlockMax) ? mb : 0;
}
size_t truncate_rel_bytes(int64_t n_max, int R, int h, int dtype) {
  const int mb = truncate_warp_mb(R, h);
  if (mb == 0 || n_max <= 0) return 0;
  const int64_t windows = (n_max + R - 1) / R;
  return (size_t)windows * win_rel_rows(mb) * 96 * elem_bytes_red(dtype);
}

// ------------------------------------------------------------------ on-chip solve
struct OcGeom {
  int mt;     // level-0 block rows (odd)
  int64_t p;  // level-0 blocks
  int G;      // CTAs
};

// The smallest odd block length (>= 3) whose CTA count fits `ctas_max`;
// a one-row tail is merged into the block before it.
template <class Tin>
static bool oc_geometry(int64_t n, int ctas_max, OcGeom& g) {
  if (n <= kBaseMax) return false;
  for (int mt = 3; mt <= oc_mt_max<Tin>(); mt += 2) {
    int64_t p = (n + mt - 1) / mt;
    if (n - (p - 1) * mt == 1) --p;
    const int64_t G = (p + kOcThreads - 1) / kOcThreads;
    if (G <= ctas_max) {
      g = {mt, p, (int)G};
      return true;
    }
  }
  return false;
}

// CTAs of k_onchip<Ar, Tin> that can be resident at once on the current
// device (at most kOcMaxCtas), found once per device; 0 if it cannot run.
// (Threads may race to fill an entry; they store the same value.)
template <class Ar, class Tin>
static int oc_ctas_max() {
  static std::atomic<int> cache[kMaxDevices];  // CTAs + 1; 0 = not known yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return 0;
  }
  const int known = cache[dev].load(std::memory_order_acquire);
  if (known > 0) return known - 1;
  int sms = 0, per = 0;
  const size_t smem = OcLayout<Ar, Tin>::kBytes;
  if (cudaFuncSetAttribute(k_onchip<Ar, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_onchip<Ar, Tin>, kOcThreads,
                                                    smem) != cudaSuccess) {
    cudaGetLastError();
    per = 0;
  }
  const int ctas = std::min(kOcMaxCtas, sms * per);
  cache[dev].store(ctas + 1, std::memory_order_release);
  return ctas;
}

// Solve the system on chip if it fits (used = true), else leave it.  xch:
// onchip_exchange_bytes() of device memory; bar: a counter (zeroed here).
template <class Ar, class Tin>
static cudaError_t launch_onchip_raw(int64_t n, const Tin* a, const Tin* b, const Tin* c,
                                     const Tin* d, Tin* x, void* xch_bytes, unsigned* bar,
                                     int* status, bool extra_arrival, cudaStream_t s,
                                     bool& used, unsigned* dmax) {
  used = false;
  OcGeom g;
  if (!oc_geometry<Tin>(n, oc_ctas_max<Ar, Tin>(), g)) return cudaSuccess;
  using T = typename Ar::T;
  T* xch = reinterpret_cast<T*>(xch_bytes);
  const uintptr_t al = (uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d | (uintptr_t)x;
  const int vec16 = (al % 16) == 0;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.G);
  cfg.blockDim = dim3(kOcThreads);
  cfg.dynamicSmemBytes = OcLayout<Ar, Tin>::kBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const unsigned arrivals = (unsigned)g.G + (extra_arrival ? 1u : 0u);
  e = cudaLaunchKernelEx(&cfg, k_onchip<Ar, Tin>, n, g.mt, g.p, a, b, c, d, x, xch, bar,
                         arrivals, status, vec16, dmax);
  if (e == cudaSuccess) used = true;
  return e;
}

// dmax: the |d / b| codes where this is level 0 (level0_dmax), else null.
template <class Ar, class Tin>
static cudaError_t launch_onchip(tps_plan_s* P, int64_t n, const Tin* a, const Tin* b,
                                 const Tin* c, const Tin* d, Tin* x, cudaStream_t s,
                                 bool& used, unsigned* dmax) {
  used = false;
  if (P->desc.flags & TPS_NO_ONCHIP) return cudaSuccess;
  return launch_onchip_raw<Ar, Tin>(n, a, b, c, d, x, P->ws + P->off_xch,
                                    reinterpret_cast<unsigned*>(P->ws + 32), P->d_status,
                                    P->test_barrier_extra, s, used, dmax);
}

unsigned* level0_dmax(tps_plan_s* P) {
  const bool on = P->desc.dtype == TPS_F64_DF ||
                  (P->desc.dtype == TPS_MIXED_F32_F64 && !P->codes_off);
  return on ? reinterpret_cast<unsigned*>(P->ws + P->off_dmax) : nullptr;
}

cudaError_t dcode_check(tps_plan_s* P, int64_t count, cudaStream_t s) {
  unsigned* dmax = level0_dmax(P);
  if (!dmax) return cudaSuccess;
  k_dcode_check<<<1, 256, 0, s>>>(dmax, count, P->d_status);
  return cudaGetLastError();
}

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

// The dynamic shared-memory limit is a per-device attribute of a kernel:
// set it once per device (bit `dev` of `done`), from any host thread.
template <class K>
static cudaError_t set_smem(K kernel, size_t smem, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Stage 1 streams chunks of K rows (or a multiple) and writes a checkpoint
// every K rows, K being Stage 3's chunk length.
#ifndef TPS_STAGE1_MUL
#define TPS_STAGE1_MUL 1  // Stage-1 chunk rows = K * TPS_STAGE1_MUL / TPS_STAGE1_DIV
#endif
#ifndef TPS_STAGE1_DIV
#define TPS_STAGE1_DIV 1
#endif
// kRef: a fused refinement step (RefineIO rf; fp64 arrays).
template <class Ar, class Tin, class Tred, int K, bool kRef = false>
static cudaError_t launch_stage1(const Level& lv, const Tin* a, const Tin* b, const Tin* c,
                                 const Tin* d, Tred* ra, Tred* rb, Tred* rc, Tred* rd, Tred* cg,
                                 Tred* cy, Tred* cv, int* status, cudaStream_t s,
                                 RefineIO rf = {}) {
  constexpr int W = kWarpsPerCta;
  constexpr int R = K * TPS_STAGE1_MUL / TPS_STAGE1_DIV;
  const size_t smem = stage1_smem_per_warp<Tin, R, kRef ? 5 : 4>() * W;
  const int64_t warps = (lv.k_end - lv.k_begin + 31) / 32;
  const unsigned grid = (unsigned)((warps + W - 1) / W);
  if (grid == 0) return cudaSuccess;
  const void* ptrs[6] = {a, b, c, d, rf.x, rf.r};
  cudaError_t e;
  if (vec16_ok<Tin>(lv.m, ptrs, kRef ? 6 : 4)) {
    static std::atomic<uint64_t> done{0};
    auto k = k_stage1<Ar, Tin, Tred, R, K, W, true, kRef>;
    if ((e = set_smem(k, smem, done)) != cudaSuccess) return e;
    k<<<grid, 32 * W, smem, s>>>(lv, a, b, c, d, ra, rb, rc, rd, cg, cy, cv, status, rf);
  } else {
    static std::atomic<uint64_t> done{0};
    auto k = k_stage1<Ar, Tin, Tred, R, K, W, false, kRef>;
    if ((e = set_smem(k, smem, done)) != cudaSuccess) return e;
    k<<<grid, 32 * W, smem, s>>>(lv, a, b, c, d, ra, rb, rc, rd, cg, cy, cv, status, rf);
  }
  return cudaGetLastError();
}

template <class Ar, class Tin, class Tred, int R, bool kRef = false>
static cudaError_t launch_stage3(const Level& lv, const Tin* a, const Tin* b, const Tin* c,
                                 const Tin* d, const Tred* xr, const Tred* cg, const Tred* cy,
                                 const Tred* cv, Tin* x, int* status, cudaStream_t s,
                                 RefineIO rf = {}) {
  constexpr int W = kWarpsPerCta;
  const size_t smem = Tile3<Tin, Tred, R, kRef ? 5 : 4>::kBytesPerWarp * W;
  const int64_t warps = (lv.k_end - lv.k_begin + 31) / 32;
  const unsigned grid = (unsigned)((warps + W - 1) / W);
  if (grid == 0) return cudaSuccess;
  const void* ptrs[5] = {a, b, c, d, x};
  cudaError_t e;
  if (vec16_ok<Tin>(lv.m, ptrs, 5)) {
    static std::atomic<uint64_t> done{0};
    auto k = k_stage3<Ar, Tin, Tred, R, W, true, kRef>;
    if ((e = set_smem(k, smem, done)) != cudaSuccess) return e;
    k<<<grid, 32 * W, smem, s>>>(lv, a, b, c, d, xr, cg, cy, cv, x, status, rf);
  } else {
    static std::atomic<uint64_t> done{0};
    auto k = k_stage3<Ar, Tin, Tred, R, W, false, kRef>;
    if ((e = set_smem(k, smem, done)) != cudaSuccess) return e;
    k<<<grid, 32 * W, smem, s>>>(lv, a, b, c, d, xr, cg, cy, cv, x, status, rf);
  }
  return cudaGetLastError();
}

template <class Ar, class Tin, class Tred>
static cudaError_t run_levels(tps_plan_s* P, const std::vector<LevelPlan>& levels, size_t idx,
                              int64_t n, const Tin* a, const Tin* b, const Tin* c, const Tin* d,
                              Tin* x, cudaStream_t s) {
  if (idx == levels.size()) {
    if (n <= 0) return cudaSuccess;
    k_base<Ar, Tin, Tin><<<1, 32, 0, s>>>(n, a, b, c, d, x, nullptr, 0, P->d_status, nullptr);
    return cudaGetLastError();
  }
  bool used = false;
  cudaError_t eo = launch_onchip<Ar, Tin>(P, n, a, b, c, d, x, s, used, nullptr);
  if (eo != cudaSuccess || used) {
    if (used) {
      P->last_onchip = 2;
      P->last_levels = (int32_t)idx;  // levels launched before the on-chip solve
    }
    return eo;
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
    lv.dmax = level0_dmax(P);
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

// One fused refinement step of the mixed solve on level 0 (fp64 arrays,
// fp32 elimination): Stage 1 on the residual of x (written to r), the
// reduced solve, Stage 3 adding the correction to x and raising max2.
cudaError_t refine_step(tps_plan_s* P, const std::vector<LevelPlan>& levels, const double* a,
                        const double* b, const double* c, const double* d, double* x, double* r,
                        unsigned long long* max2, cudaStream_t s) {
  using Ar = ArF32;
  using Tin = double;
  using Tred = float;
  constexpr int R = kChunkRows<Tin>;
  const LevelPlan& L = levels[0];
  const RefineIO rf{x, r, max2};
  Tred* red[5];
  for (int i = 0; i < 5; ++i) red[i] = reinterpret_cast<Tred*>(P->ws + L.off_red[i]);
  Tred* ck[3];
  for (int i = 0; i < 3; ++i) ck[i] = reinterpret_cast<Tred*>(P->ws + L.off_ck[i]);
  Level lv = L.lv;
  lv.k_begin = 0;
  lv.k_end = lv.p;
  lv.dmax = nullptr;  // a residual's range codes are not judged
  cudaError_t e = cudaMemsetAsync(max2, 0, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess)
    e = launch_stage1<Ar, Tin, Tred, R, true>(lv, a, b, c, d, red[0], red[1], red[2], red[3],
                                              ck[0], ck[1], ck[2], P->d_status, s, rf);
  if (e == cudaSuccess) e = reduced_solve(P, levels, s);
  if (e == cudaSuccess)
    e = launch_stage3<Ar, Tin, Tred, R, true>(lv, a, b, c, r, red[4], ck[0], ck[1], ck[2], x,
                                              P->d_status, s, rf);
  return e;
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
                                          (const Tin*)d, (Tin*)x, bnd, nbnd, P->d_status,
                                          level0_dmax(P));
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
    P->graph_onchip = P->last_onchip;
    P->graph_levels = P->last_levels;
  }
  P->last_onchip = P->graph_onchip;
  P->last_levels = P->graph_levels;
  return cudaGraphLaunch(P->graph, s);
}

static tps_status run_solve_direct(tps_plan_s* P, int64_t n, const void* a, const void* b,
                                   const void* c, const void* d, void* x, cudaStream_t s,
                                   const std::vector<LevelPlan>& lv, cudaEvent_t* ev,
                                   const int64_t* bnd, int64_t nbnd);

// TPS_GRAPH without stage events: capture the whole solve on the plan's
// private stream the first time a geometry and set of pointers is seen,
// then replay it as one graph launch.  Everything the captured launches
// read from the host (sizes, pointers, the level plan) is in the key.
static tps_status run_solve_graph(tps_plan_s* P, int64_t n, const void* a, const void* b,
                                  const void* c, const void* d, void* x, cudaStream_t s,
                                  const std::vector<LevelPlan>& lv, const int64_t* bnd,
                                  int64_t nbnd) {
  const int64_t key[16] = {n, (int64_t)a, (int64_t)b, (int64_t)c, (int64_t)d, (int64_t)x,
                           (int64_t)bnd, nbnd, P->m, P->m_reduced, (int64_t)lv.size(),
                           (int64_t)P->ws, P->desc.dtype, (int64_t)P->desc.flags, 0, 0};
  bool same = P->solve_graph != nullptr;
  for (int i = 0; i < 16 && same; ++i) same = P->sgkey[i] == key[i];
  if (!same) {
    if (P->solve_graph) {
      cudaGraphExecDestroy(P->solve_graph);
      P->solve_graph = nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!P->cap_stream) e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return TPS_ERR_CUDA;
    const tps_status st = run_solve_direct(P, n, a, b, c, d, x, P->cap_stream, lv, nullptr, bnd,
                                           nbnd);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(P->cap_stream, &g);
    if (st != TPS_OK || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return st != TPS_OK ? st : TPS_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&P->solve_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      P->solve_graph = nullptr;
      return TPS_ERR_CUDA;
    }
    for (int i = 0; i < 16; ++i) P->sgkey[i] = key[i];
    P->sg_onchip = P->last_onchip;
    P->sg_levels = P->last_levels;
  }
  P->last_onchip = P->sg_onchip;
  P->last_levels = P->sg_levels;
  return cudaGraphLaunch(P->solve_graph, s) == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}

tps_status run_solve(tps_plan_s* P, int64_t n, const void* a, const void* b, const void* c,
                     const void* d, void* x, cudaStream_t s, const std::vector<LevelPlan>& lv,
                     cudaEvent_t* ev, const int64_t* bnd, int64_t nbnd) {
  if ((P->desc.flags & TPS_GRAPH) && !ev && P->desc.dtype != TPS_MIXED_F32_F64)
    return run_solve_graph(P, n, a, b, c, d, x, s, lv, bnd, nbnd);
  return run_solve_direct(P, n, a, b, c, d, x, s, lv, ev, bnd, nbnd);
}

static tps_status run_solve_direct(tps_plan_s* P, int64_t n, const void* a, const void* b,
                                   const void* c, const void* d, void* x, cudaStream_t s,
                                   const std::vector<LevelPlan>& lv, cudaEvent_t* ev,
                                   const int64_t* bnd, int64_t nbnd) {
  cudaError_t e = cudaSuccess;
  P->last_onchip = 0;
  if (ev) e = cudaEventRecord(ev[0], s);
  bool onchip = false;
  if (e == cudaSuccess && !lv.empty() && nbnd == 0) {  // the whole system on chip
    e = dispatch(P->desc.dtype, [&](auto ar, auto* tin, auto* tred) -> cudaError_t {
      using Ar = decltype(ar);
      using Tin = std::remove_pointer_t<decltype(tin)>;
      (void)tred;
      return launch_onchip<Ar, Tin>(P, n, (const Tin*)a, (const Tin*)b, (const Tin*)c,
                                    (const Tin*)d, (Tin*)x, s, onchip, level0_dmax(P));
    });
    if (onchip) {
      P->last_onchip = 1;
      P->last_levels = 0;
    }
  }
  if (onchip) {
    for (int i = 1; i < 3 && e == cudaSuccess && ev; ++i) e = cudaEventRecord(ev[i], s);
  } else if (lv.empty()) {
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = base_solve(P, n, a, b, c, d, x, s, bnd, nbnd);
    if (e == cudaSuccess) e = dcode_check(P, nbnd + 1, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
  } else {
    if (e == cudaSuccess) e = stage1_range(P, lv[0], 0, lv[0].lv.p, a, b, c, d, s);
    if (e == cudaSuccess) e = dcode_check(P, nbnd + 1, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    // with stage events (TPS_TRACE) TPS_GRAPH captures Stage 2 alone; without
    // them the whole solve is one graph already (run_solve_graph)
    if (e == cudaSuccess)
      e = ((P->desc.flags & TPS_GRAPH) && ev) ? reduced_solve_graph(P, lv, s)
                                              : reduced_solve(P, lv, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
    if (e == cudaSuccess) e = stage3_range(P, lv[0], 0, lv[0].lv.p, a, b, c, d, x, s);
  }
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], s);
  return e == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}

// ------------------------------------------------------------------ windowed solve
template <class Ar, class Tin>
static cudaError_t launch_window(tps_plan_s* P, int64_t n, const Tin* a, const Tin* b,
                                 const Tin* c, const Tin* d, Tin* x, cudaStream_t s) {
  static std::atomic<uint64_t> done{0};  // the attribute allows the largest window
  cudaError_t e = set_smem(k_window<Ar, Tin>, WinLayout<Ar, Tin>::bytes(kWinRowsMax), done);
  if (e != cudaSuccess) return e;
  const int R = P->m, h = P->m_reduced;
  const size_t smem = WinLayout<Ar, Tin>::bytes(R + 2 * h);  // this window size
  const int64_t windows = (n + R - 1) / R;
  const uintptr_t al = (uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d | (uintptr_t)x;
  unsigned* bound = reinterpret_cast<unsigned*>(P->ws + 8);
  e = cudaMemsetAsync(bound, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const float tol = (float)(P->desc.tol > 0.0 ? P->desc.tol : 1e-12);
  k_window<Ar, Tin><<<(unsigned)windows, kWinThreads, smem, s>>>(
      n, R, h, a, b, c, d, x, tol, bound, P->d_status, (al % 16) == 0, level0_dmax(P));
  return cudaGetLastError();
}

// One warp per window (k_wsolve): R + 2 h = 32 mb.
template <class Ar, class Tin, class Tred>
static cudaError_t launch_wsolve(tps_plan_s* P, int64_t n, int mb, const Tin* a, const Tin* b,
                                 const Tin* c, const Tin* d, Tin* x, cudaStream_t s) {
  using T = typename Ar::T;
  const int R = P->m, h = P->m_reduced;
  constexpr int kVec = 16 / (int)sizeof(Tin);
  const uintptr_t al = (uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d | (uintptr_t)x;
  const bool vec = (al % 16) == 0 && mb % kVec == 0 && R % kVec == 0 && h % kVec == 0;
  unsigned* bound = reinterpret_cast<unsigned*>(P->ws + 8);
  cudaError_t e = cudaMemsetAsync(bound, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const float tol = (float)(P->desc.tol > 0.0 ? P->desc.tol : 1e-12);
  Tred* rel = reinterpret_cast<Tred*>(P->ws + P->off_rel);
  const unsigned windows = (unsigned)((n + R - 1) / R);
  constexpr size_t smem = WinSmem<Tin, Tred, T>::kBytes;
  if (vec)
    k_wsolve<Ar, Tin, Tred, true><<<windows, 32, smem, s>>>(n, R, h, mb, a, b, c, d, x, rel, tol,
                                                            bound, P->d_status, level0_dmax(P));
  else
    k_wsolve<Ar, Tin, Tred, false><<<windows, 32, smem, s>>>(n, R, h, mb, a, b, c, d, x, rel, tol,
                                                             bound, P->d_status, level0_dmax(P));
  return cudaGetLastError();
}

tps_status run_truncated(tps_plan_s* P, int64_t n, const void* a, const void* b, const void* c,
                         const void* d, void* x, cudaStream_t s) {
  P->last_onchip = 0;
  P->last_levels = 0;
  cudaError_t e = cudaSuccess;
  const int mb = truncate_warp_mb(P->m, P->m_reduced);
  if (n <= kBaseMax) {
    e = base_solve(P, n, a, b, c, d, x, s, nullptr, 0);
  } else if (mb > 0) {
    e = dispatch(P->desc.dtype, [&](auto ar, auto* tin, auto* tred) -> cudaError_t {
      using Ar = decltype(ar);
      using Tin = std::remove_pointer_t<decltype(tin)>;
      using Tred = std::remove_pointer_t<decltype(tred)>;
      return launch_wsolve<Ar, Tin, Tred>(P, n, mb, (const Tin*)a, (const Tin*)b, (const Tin*)c,
                                          (const Tin*)d, (Tin*)x, s);
    });
  } else {
    e = dispatch(P->desc.dtype, [&](auto ar, auto* tin, auto* tred) -> cudaError_t {
      using Ar = decltype(ar);
      using Tin = std::remove_pointer_t<decltype(tin)>;
      (void)tred;
      return launch_window<Ar, Tin>(P, n, (const Tin*)a, (const Tin*)b, (const Tin*)c,
                                    (const Tin*)d, (Tin*)x, s);
    });
  }
  if (e == cudaSuccess) e = dcode_check(P, 1, s);
  return e == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}


cudaError_t onchip_solve(int dtype, int64_t n, const void* a, const void* b, const void* c,
                         const void* d, void* x, void* xch, unsigned* bar, int* status,
                         cudaStream_t s, bool& used, unsigned* dmax) {
  return dispatch(dtype, [&](auto ar, auto* tin, auto* tred) -> cudaError_t {
    using Ar = decltype(ar);
    using Tin = std::remove_pointer_t<decltype(tin)>;
    (void)tred;
    return launch_onchip_raw<Ar, Tin>(n, (const Tin*)a, (const Tin*)b, (const Tin*)c,
                                      (const Tin*)d, (Tin*)x, xch, bar, status, false, s, used,
                                      dmax);
  });
}

}  // namespace tps
