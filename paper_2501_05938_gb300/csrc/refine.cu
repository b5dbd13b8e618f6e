// Mixed-precision iterative refinement (TPS_MIXED_F32_F64): the partition
// elimination runs in binary32 (fp64 inputs split to fp32 on load), while
// the residual r = d - A x and the update x += delta stay in fp64:
//
//   x_0 = solve_f32(A, d)
//   repeat: r = d - A x (fp64); delta = solve_f32(A, r); x += delta (fp64)
//   until max|delta| <= tol * max|x|, or max_iters corrections.
//
// (Classical iterative refinement, Wilkinson 1963 / Moler 1967.)  The
// stopping test reads two fp64 maxima back to the host after every
// correction, so a mixed-precision solve synchronises its stream once per
// iteration.
//
// Where the system is solved level by level (every size but those the
// single-launch on-chip solve takes), a correction is one pass of the
// partition method over the rows (refine_step): Stage 1 forms the residual
// from the rows and x as it streams them and writes it out, Stage 3 reads
// the residual back as its right-hand side and adds its result to x.  Per
// row that moves a, b, c, d, x in and r out, then a, b, c, r, x in and x
// out: 96 bytes against 144 for a residual pass, a solve and an update pass.
// The on-chip route keeps the three separate passes below.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "tps_internal.h"

namespace tps {

namespace {

// Is row i the first row of a packed system (other than the first)?
__device__ __forceinline__ bool is_start(const int64_t* bnd, int64_t nbnd, int64_t i) {
  if (nbnd == 0) return false;
  const int64_t j = Bounds::lower(bnd, nbnd, i);
  return j < nbnd && bnd[j] == i;
}

// r = d - A x in fp64, couplings cut at packed-system boundaries.
__global__ void k_residual(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                           const double* __restrict__ c, const double* __restrict__ d,
                           const double* __restrict__ x, double* __restrict__ r,
                           const int64_t* __restrict__ bnd, int64_t nbnd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool first = i == 0 || is_start(bnd, nbnd, i);
    const bool last = i == n - 1 || is_start(bnd, nbnd, i + 1);
    double s = b[i] * x[i];
    if (!first) s = fma(a[i], x[i - 1], s);
    if (!last) s = fma(c[i], x[i + 1], s);
    r[i] = d[i] - s;
  }
}

// x += delta in fp64; maxima of |delta| and |x| (non-negative doubles order
// like their bit patterns, so an integer atomicMax serves).
__global__ void k_update(int64_t n, double* __restrict__ x, const double* __restrict__ delta,
                         unsigned long long* __restrict__ maxima) {
  double md = 0.0, mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double dv = delta[i];
    const double xv = x[i] + dv;
    x[i] = xv;
    md = fmax(md, fabs(dv));
    mx = fmax(mx, fabs(xv));
  }
  for (int o = 16; o > 0; o >>= 1) {
    md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    // NaN compares false everywhere: record it as +inf so it cannot pass
    if (!(md == md)) md = __longlong_as_double(0x7FF0000000000000ll);
    atomicMax(&maxima[0], (unsigned long long)__double_as_longlong(md));
    atomicMax(&maxima[1], (unsigned long long)__double_as_longlong(mx));
  }
}

unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

tps_status run_refine(tps_plan_s* P, int64_t n, const double* a, const double* b,
                      const double* c, const double* d, double* x, cudaStream_t s,
                      const std::vector<LevelPlan>& lv, const int64_t* bnd, int64_t nbnd) {
  double* r = reinterpret_cast<double*>(P->ws + P->off_refine);
  double* dl = reinterpret_cast<double*>(P->ws + P->off_refine + align_up((size_t)n * 8));
  unsigned long long* maxima = reinterpret_cast<unsigned long long*>(P->d_scalars);
  const int max_iters = P->desc.max_iters > 0 ? P->desc.max_iters : 10;
  const double tol = P->desc.tol > 0.0 ? P->desc.tol : 1e-12;
  P->last_iters = 0;
  P->last_corr = 0.0;
  P->last_refine_fused = 0;
  // the first solve carries the range codes of the system (an fp32 x0 of a
  // right-hand side below the pairs' range would be 0 and 'converge'); the
  // corrections' right-hand sides are small by construction and skip them
  struct CodesOn {
    tps_plan_s* P;
    ~CodesOn() { P->codes_off = false; }
  } restore{P};
  P->codes_off = false;
  tps_status st = run_solve(P, n, a, b, c, d, x, s, lv, nullptr, bnd, nbnd);
  if (st != TPS_OK) return st;
  P->codes_off = true;
  // the fused step where level 0 runs as separate Stage 1 / Stage 3 sweeps
  const bool fused = !lv.empty() && P->last_onchip != 1 && !P->test_unfused_refine;
  P->last_refine_fused = fused ? 1 : 0;
  for (int it = 1; it <= max_iters; ++it) {
    if (fused) {
      if (refine_step(P, lv, a, b, c, d, x, r, maxima, s) != cudaSuccess) return TPS_ERR_CUDA;
    } else {
      k_residual<<<grid_for(n), 256, 0, s>>>(n, a, b, c, d, x, r, bnd, nbnd);
      if (cudaGetLastError() != cudaSuccess) return TPS_ERR_CUDA;
      st = run_solve(P, n, a, b, c, r, dl, s, lv, nullptr, bnd, nbnd);
      if (st != TPS_OK) return st;
      if (cudaMemsetAsync(maxima, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess)
        return TPS_ERR_CUDA;
      k_update<<<grid_for(n), 256, 0, s>>>(n, x, dl, maxima);
    }
    unsigned long long h[2];
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h, maxima, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return TPS_ERR_CUDA;
    double md, mx;
    std::memcpy(&md, &h[0], sizeof(double));
    std::memcpy(&mx, &h[1], sizeof(double));
    P->last_iters = it;
    P->last_corr = mx > 0.0 ? md / mx : md;
    if (md <= tol * mx) return TPS_OK;
  }
  P->host_status = TPS_ERR_NO_CONVERGENCE;
  return TPS_OK;
}

}  // namespace tps
