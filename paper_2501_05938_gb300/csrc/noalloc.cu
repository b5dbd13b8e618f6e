// tps_solve_noalloc: the device-resident partition solve for callers that
// must not allocate device memory -- for example code under a framework
// that owns every device allocation through its own caching allocator, code
// running under a fixed device-memory budget, or latency-critical loops
// where a cudaMalloc (which may synchronise the device) is not acceptable.
// Instead of a plan and its workspace, this entry point keeps
// its scratch (the reduced systems, the Stage-1 checkpoints and a status
// word; or, when the system fits on chip and is solved by one cooperative
// launch, that launch's barrier counter and exchange rows) in one
// fixed-size array in device global memory, declared at file scope below.  Every GPU that loads the library holds that array
// (kScratchBytes) until the process exits.  All calls share it, and it keeps
// whatever the last call left there; so two calls whose work overlaps on
// the GPU (different streams, or different host threads) race on it and
// must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>

#include "tps_internal.h"

namespace {

using namespace tps;

constexpr int64_t kMaxRows = TPS_NOALLOC_MAX_ROWS;
constexpr int kM0 = 64;           // rows per block at the top level
constexpr int kMr = 32;           // rows per block at the reduced levels
constexpr int kMaxLevels = 8;
constexpr size_t kScratchBytes = size_t(2) << 20;  // 2 MiB per GPU

// The scratch array.  In host code `g_scratch` names a host-side shadow,
// not device memory: its device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, looked up once per device with that device
// current (the first call on a device does it).
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

tps_status scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TPS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return TPS_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return TPS_OK;
}

// Level layout inside the scratch, on the stack (no host allocation either).
struct Layout {
  LevelPlan lv[kMaxLevels];
  int levels = 0;
  size_t bytes = 0;
};

bool make_layout(int64_t n, size_t top_elem, size_t red_elem, Layout& L) {
  size_t off = align_up(64);  // status word first
  int64_t N = n;
  size_t elem = top_elem;
  int m = kM0;
  L.levels = 0;
  while (N > kBaseMax) {
    if (L.levels == kMaxLevels) return false;
    LevelPlan& P = L.lv[L.levels++];
    P = LevelPlan{};
    P.R = chunk_rows(elem);
    P.lv = make_level(N, m, P.R);
    const int64_t nr = 2 * P.lv.p;
    for (int i = 0; i < 5; ++i) {
      P.off_red[i] = off;
      off = align_up(off + (size_t)nr * red_elem);
    }
    const size_t nck = (size_t)P.lv.ncap * (size_t)P.lv.p;
    for (int i = 0; i < 3; ++i) {
      P.off_ck[i] = off;
      off = align_up(off + nck * red_elem);
    }
    N = nr;
    elem = red_elem;
    m = kMr;
  }
  L.bytes = off;
  return off <= kScratchBytes;
}

template <class Tin>
bool aligned16(int m, const void* const* p, int k) {
  if (m % (16 / (int)sizeof(Tin))) return false;
  for (int i = 0; i < k; ++i)
    if ((uintptr_t)p[i] % 16) return false;
  return true;
}

// dmax: the system's range codes at level 0 of a double-float solve (zero
// before the call, zero again after it), else null.
template <class Ar, class Tin, class Tred>
cudaError_t run(unsigned char* ws, const Layout& L, int idx, int64_t n, const Tin* a,
                const Tin* b, const Tin* c, const Tin* d, Tin* x, int* st, cudaStream_t s,
                unsigned* dmax) {
  if (idx == L.levels) {
    k_base<Ar, Tin, Tin><<<1, 32, 0, s>>>(n, a, b, c, d, x, nullptr, 0, st, dmax);
    if (dmax) k_dcode_check<<<1, 256, 0, s>>>(dmax, 1, st);
    return cudaGetLastError();
  }
  const LevelPlan& P = L.lv[idx];
  constexpr int K = kChunkRows<Tin>;  // Stage-3 chunk rows, checkpoint spacing (as make_layout)
  constexpr int R1 = K;
  Level lv = P.lv;
  lv.dmax = dmax;
  Tred* red[5];
  for (int i = 0; i < 5; ++i) red[i] = reinterpret_cast<Tred*>(ws + P.off_red[i]);
  Tred* ck[3];
  for (int i = 0; i < 3; ++i) ck[i] = reinterpret_cast<Tred*>(ws + P.off_ck[i]);
  const unsigned grid = (unsigned)((P.lv.p + 31) / 32);
  const void* in4[4] = {a, b, c, d};
  const void* in5[5] = {a, b, c, d, x};
  if (aligned16<Tin>(P.lv.m, in4, 4))
    k_stage1<Ar, Tin, Tred, R1, K, 1, true><<<grid, 32, stage1_smem_per_warp<Tin, R1>(), s>>>(
        lv, a, b, c, d, red[0], red[1], red[2], red[3], ck[0], ck[1], ck[2], st);
  else
    k_stage1<Ar, Tin, Tred, R1, K, 1, false><<<grid, 32, stage1_smem_per_warp<Tin, R1>(), s>>>(
        lv, a, b, c, d, red[0], red[1], red[2], red[3], ck[0], ck[1], ck[2], st);
  if (dmax) k_dcode_check<<<1, 256, 0, s>>>(dmax, 1, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = run<Ar, Tred, Tred>(ws, L, idx + 1, 2 * P.lv.p, red[0], red[1], red[2], red[3], red[4],
                          st, s, nullptr);
  if (e != cudaSuccess) return e;
  if (aligned16<Tin>(P.lv.m, in5, 5))
    k_stage3<Ar, Tin, Tred, K, 1, true><<<grid, 32, Tile3<Tin, Tred, K>::kBytesPerWarp, s>>>(
        P.lv, a, b, c, d, red[4], ck[0], ck[1], ck[2], x, st);
  else
    k_stage3<Ar, Tin, Tred, K, 1, false><<<grid, 32, Tile3<Tin, Tred, K>::kBytesPerWarp, s>>>(
        P.lv, a, b, c, d, red[4], ck[0], ck[1], ck[2], x, st);
  return cudaGetLastError();
}

// Translate the status bits into a tps_status for the caller's output.
__global__ void k_report(const int* st, int32_t* out) {
  const int w = *st;
  *out = (w & ST_BAD_PIVOT) ? TPS_ERR_ZERO_PIVOT
         : (w & ST_TIMEOUT) ? TPS_ERR_TIMEOUT
         : (w & ST_RANGE)   ? TPS_ERR_RANGE
                            : TPS_OK;
}

// A cooperative launch the device refuses for its size or resources (fewer
// SMs than the cached occupancy assumed, e.g. under an SM partition):
// the level-by-level route serves instead.
bool launch_refused(cudaError_t e) {
  return e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorLaunchOutOfResources ||
         e == cudaErrorInvalidConfiguration;
}

bool overlap(const void* p, const void* q, size_t bytes) {
  const uintptr_t u = (uintptr_t)p, v = (uintptr_t)q;
  return u < v + bytes && v < u + bytes;
}

}  // namespace

extern "C" tps_status tps_solve_noalloc(int32_t dtype, int64_t n, const void* a, const void* b,
                                        const void* c, const void* d, void* x,
                                        int32_t* status_out, void* stream) {
  if (dtype != TPS_F64 && dtype != TPS_F64_DF && dtype != TPS_F32) return TPS_ERR_INVALID_ARG;
  if (n < 0 || n > kMaxRows) return TPS_ERR_INVALID_ARG;
  if (n == 0) return TPS_OK;
  const size_t es = dtype == TPS_F32 ? 4 : 8;
  const void* in[4] = {a, b, c, d};
  for (const void* p : in)
    if (!p || (uintptr_t)p % es || overlap(p, x, (size_t)n * es)) return TPS_ERR_INVALID_ARG;
  if (!x || (uintptr_t)x % es || (status_out && (uintptr_t)status_out % 4))
    return TPS_ERR_INVALID_ARG;
  Layout L;
  if (!make_layout(n, es, es, L)) return TPS_ERR_INVALID_ARG;
  unsigned char* ws = nullptr;
  tps_status ts = scratch_address(&ws);
  if (ts != TPS_OK) return ts;
  cudaStream_t s = (cudaStream_t)stream;
  int* st = reinterpret_cast<int*>(ws);
  // the first 64 bytes (status word, on-chip barrier counter, the three
  // range codes at 40) are the only scratch that must start from zero; the
  // reduced systems and checkpoints are fully rewritten by every call
  unsigned* dmax = dtype == TPS_F64_DF ? reinterpret_cast<unsigned*>(ws + 40) : nullptr;
  cudaError_t e = cudaMemsetAsync(st, 0, 64, s);
  // the whole system in one on-chip launch where it fits (its barrier
  // counter and exchange rows sit where the levels would go); a test switch
  // (TPS_TEST_NOALLOC_LEVELS=1) keeps the level-by-level route
  bool onchip = false;
  const char* lvl = std::getenv("TPS_TEST_NOALLOC_LEVELS");
  if (e == cudaSuccess && !(lvl && lvl[0] == '1')) {
    e = onchip_solve(dtype, n, a, b, c, d, x, ws + align_up(64),
                     reinterpret_cast<unsigned*>(ws + 32), st, s, onchip, dmax);
    if (e != cudaSuccess && launch_refused(e)) {
      cudaGetLastError();
      e = cudaSuccess;
      onchip = false;
    }
  }
  if (e == cudaSuccess && !onchip) {
    switch (dtype) {
      case TPS_F64:
        e = run<ArF64, double, double>(ws, L, 0, n, (const double*)a, (const double*)b,
                                       (const double*)c, (const double*)d, (double*)x, st, s,
                                       nullptr);
        break;
      case TPS_F64_DF:
        e = run<ArDF, double, float2>(ws, L, 0, n, (const double*)a, (const double*)b,
                                      (const double*)c, (const double*)d, (double*)x, st, s,
                                      dmax);
        break;
      default:
        e = run<ArF32, float, float>(ws, L, 0, n, (const float*)a, (const float*)b,
                                     (const float*)c, (const float*)d, (float*)x, st, s,
                                     nullptr);
        break;
    }
  }
  if (e == cudaSuccess && status_out) {
    k_report<<<1, 1, 0, s>>>(st, status_out);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}
