// Scale-free pieces of the truncated decoupling's per-window error bound
// (TPS_TRUNCATE), shared by the one-CTA and the one-warp window kernels.
#pragma once
#include <cuda_runtime.h>

#include "arith.cuh"

namespace tps {

// A row's dominance ratio (|a| + |c|) / |b|, rounded up, in binary32.  fp64
// rows are first scaled by their diagonal's power of two with integer
// operations (split_row), so a row anywhere in the fp64 range gives its
// ratio (the conversion instructions would also run on the slow fp64 pipe);
// the parts are truncated (up to 2^-23 low), which the caller's 2^-20
// widening of q covers.
__device__ __forceinline__ float win_row_q(double a, double b, double c) {
  df64 A, B, C, D;
  RowChk k;
  split_row<false>(a, b, c, 0.0, A, B, C, D, k);
  return __fdiv_ru(__fadd_ru(fabsf(A.hi), fabsf(C.hi)), fabsf(B.hi));
}
__device__ __forceinline__ float win_row_q(float a, float b, float c) {
  return __fdiv_ru(__fadd_ru(fabsf(a), fabsf(c)), fabsf(b));
}
// |v| as an ordered integer key (high word of fp64, all of fp32); the value
// with the key's bits (low word 0) is a lower bound on |v|
__device__ __forceinline__ unsigned mag_key(double v) {
  return (unsigned)__double2hiint(v) & 0x7FFFFFFFu;
}
__device__ __forceinline__ unsigned mag_key(float v) { return __float_as_uint(v) & 0x7FFFFFFFu; }

}  // namespace tps
