// Seeded synthetic tridiagonal systems on the device.  Same definition as
// the numpy generator in synth/__init__.py (SplitMix64 counters, the "paper"
// and "ratio" diagonals, d = A x_true with every product and sum rounded
// once); the two produce bit-identical arrays.  Input synthesis only: no
// solver arithmetic lives here.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double unif(uint64_t key, int64_t i) {
  const uint64_t z = mix64(key + (uint64_t)(i + 1) * kGolden);
  return __dmul_rn(__ull2double_rn(z >> 11), 0x1.0p-53);
}

__device__ __forceinline__ double sym(uint64_t key, int64_t i) {
  return __dadd_rn(__dmul_rn(2.0, unif(key, i)), -1.0);
}

struct Keys {
  uint64_t a, b, c, x;
};

__global__ void k_synth(int64_t n, const int64_t* __restrict__ offsets, int64_t count, int kind,
                        double ratio, Keys K, double* __restrict__ a, double* __restrict__ b,
                        double* __restrict__ c, double* __restrict__ d, double* __restrict__ xt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    bool first, last;
    if (offsets) {
      int64_t lo = 0, hi = count - 1;  // largest s with offsets[s] <= i
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= i) lo = mid; else hi = mid - 1;
      }
      first = (i == offsets[lo]);
      last = (i == offsets[lo + 1] - 1);
    } else {
      first = (i == 0);
      last = (i == n - 1);
    }
    const double av = first ? 0.0 : sym(K.a, i);
    const double cv = last ? 0.0 : sym(K.c, i);
    double bv;
    const double off = __dadd_rn(fabs(av), fabs(cv));
    if (kind == 0) {
      bv = __dadd_rn(off, __dadd_rn(1.0, unif(K.b, i)));
    } else {
      bv = __dmul_rn(ratio, fmax(off, 0x1.0p-20));
    }
    const double xv = sym(K.x, i);
    const double ta = first ? 0.0 : __dmul_rn(av, sym(K.x, i - 1));
    const double tc = last ? 0.0 : __dmul_rn(cv, sym(K.x, i + 1));
    a[i] = av;
    b[i] = bv;
    c[i] = cv;
    xt[i] = xv;
    d[i] = __dadd_rn(__dadd_rn(ta, __dmul_rn(bv, xv)), tc);
  }
}

}  // namespace

extern "C" int tps_synth_system(uint64_t seed, int64_t n, const int64_t* offsets, int64_t count,
                                int kind, double ratio, double* a, double* b, double* c,
                                double* d, double* x_true, void* stream) {
  if (n < 0 || (offsets && count < 1) || (kind != 0 && kind != 1)) return 1;
  if (n == 0) return 0;
  Keys K;
  K.a = mix64(seed + 1 * kGolden);
  K.b = mix64(seed + 2 * kGolden);
  K.c = mix64(seed + 3 * kGolden);
  K.x = mix64(seed + 4 * kGolden);
  const int threads = 256;
  int64_t blocks = (n + threads - 1) / threads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_synth<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(n, offsets, count, kind, ratio,
                                                                  K, a, b, c, d, x_true);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
