// Measured fp64 instruction rates of the current device: the denominator
// of the plain (native fp64) solve's roofline, for which no published
// figure of this part is at hand.  Every thread runs independent chains of
// one fp64 operation (fused multiply-add, multiply or add), at two
// occupancies, enough chains per SM to cover the pipe's latency; the best
// launch of each kind counts.
#include <cuda_runtime.h>

#include "tps_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kIters = 2048;

// kind 0: v = v * m + c; 1: v = v * m; 2: v = v + c
template <int kKind, int kChains>
__global__ void __launch_bounds__(kThreads) k_fp64_op(double* __restrict__ out, int iters) {
  double v[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) v[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
  // operands in registers (not constants), as in the solver's kernels
  const double mul = 0.9999999 + 1e-13 * (double)(threadIdx.x & 3);
  const double add = 1e-9 * (double)(1 + (threadIdx.x & 1));
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if constexpr (kKind == 0) v[k] = fma(v[k], mul, add);
      else if constexpr (kKind == 1) v[k] = __dmul_rn(v[k], mul);
      else v[k] = __dadd_rn(v[k], add);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += v[k];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

// operations per second of one kernel configuration, best of 5 launches
template <int kKind, int kChains>
cudaError_t rate(double* out, unsigned blocks, cudaEvent_t e0, cudaEvent_t e1, double& best) {
  k_fp64_op<kKind, kChains><<<blocks, kThreads>>>(out, kIters);  // warm-up
  for (int r = 0; r < 5; ++r) {
    float ms = 0.0f;
    cudaEventRecord(e0);
    k_fp64_op<kKind, kChains><<<blocks, kThreads>>>(out, kIters);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) return e;
    const double v = (double)blocks * kThreads * kChains * kIters / (ms * 1e-3);
    if (v > best) best = v;
  }
  return cudaSuccess;
}

template <int kKind>
cudaError_t kind_rate(double* out, int sms, cudaEvent_t e0, cudaEvent_t e1, double& best) {
  best = 0.0;
  cudaError_t e = rate<kKind, 8>(out, (unsigned)(4 * sms), e0, e1, best);
  if (e == cudaSuccess) e = rate<kKind, 16>(out, (unsigned)(8 * sms), e0, e1, best);
  return e;
}

}  // namespace

extern "C" tps_status tps_measure_fp64_rates(double* fma_per_s, double* mul_per_s,
                                             double* add_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TPS_ERR_CUDA;
  double* out = nullptr;
  if (cudaMalloc(&out, (size_t)8 * sms * kThreads * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return TPS_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double r[3] = {0.0, 0.0, 0.0};
  if (e == cudaSuccess) e = kind_rate<0>(out, sms, e0, e1, r[0]);
  if (e == cudaSuccess) e = kind_rate<1>(out, sms, e0, e1, r[1]);
  if (e == cudaSuccess) e = kind_rate<2>(out, sms, e0, e1, r[2]);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TPS_ERR_CUDA;
  }
  if (fma_per_s) *fma_per_s = r[0];
  if (mul_per_s) *mul_per_s = r[1];
  if (add_per_s) *add_per_s = r[2];
  return TPS_OK;
}
