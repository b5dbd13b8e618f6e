// Single-pass, on-chip partition solve for systems that fit in the GPU's
// shared memory (the same method as the multi-launch path: Sec. 1 and
// Sec. 2.2 of the paper, blocks eliminated onto their first and last rows,
// a reduced interface system, per-block recovery), as ONE cooperative
// launch that reads a, b, c, d from HBM once and writes x once.
//
//   CTA c owns the consecutive level-0 blocks [c*T, (c+1)*T) of mt rows
//   (T = 256 threads, one block per thread; mt odd, so a thread's rows start
//   on a different bank than its neighbour's) and loads their rows into
//   shared memory.
//   Stage 1, level 0: every thread eliminates its block; the normalised
//   relation x_j = g'_j - alpha'_j f - c'_j x_{j+1} of each interior row
//   overwrites that row's a, b, c in place, and the block's two reduced
//   rows go to the CTA's level-1 arrays.
//   Stage 1, levels 1..: the CTA's reduced system (2 rows per block, still
//   coupled to the neighbouring CTAs only through its first and last row)
//   is eliminated the same way in 8-row blocks, in shared memory, until one
//   block of at most 8 rows is left; its two reduced rows -- the CTA's
//   interface equations -- go to global memory.
//   One grid barrier (bounded wait; a timeout sets ST_TIMEOUT and every CTA
//   returns).
//   Stage 2: every CTA reads the 2G interface rows and solves them by
//   parallel cyclic reduction (redundantly, so no second barrier).
//   Stage 3: down the levels, every block back-substitutes from its two
//   interface values through the stored relations; level 0 leaves x in the
//   d slots, which go out to global memory in 16-byte pieces.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "partition_kernels.cuh"
#include "window_bound.cuh"

namespace tps {

constexpr int kOcThreads = 256;                 // threads per CTA = level-0 blocks per CTA
constexpr int kOcMaxCtas = 160;                 // interface rows <= 2 * this
constexpr int kOcBlock = 8;                     // block rows at the intra-CTA levels >= 1
constexpr int kOcFinal = 8;                     // last intra-CTA block: at most this many rows
constexpr int kOcLevelRows = 512 + 128 + 32 + 8;  // levels 1..4 for 2 * kOcThreads rows
constexpr int kOcLevelSlots = kOcLevelRows + kOcLevelRows / kOcBlock + kOcBlock;
constexpr unsigned kOcSpinLimit = 1u << 22;     // grid barrier: polls of ~100 ns each

template <class Tin>
constexpr int oc_mt_max() {  // largest level-0 block (odd)
  return sizeof(Tin) >= 8 ? 23 : 47;
}
template <class Tin>
constexpr int oc_rows_max() {  // level-0 rows of one CTA (one merged one-row tail)
  return kOcThreads * oc_mt_max<Tin>() + 1;
}

// Shared-memory layout: level-0 arrays (Tin), level arrays (T), interface
// system (T); each part 16-byte aligned.
template <class Ar, class Tin>
struct OcLayout {
  using T = typename Ar::T;
  static constexpr size_t kL0 = ((size_t)oc_rows_max<Tin>() * sizeof(Tin) + 15) / 16 * 16;
  static constexpr size_t kLv = ((size_t)kOcLevelSlots * sizeof(T) + 15) / 16 * 16;
  static constexpr size_t kPc = ((size_t)2 * kOcMaxCtas * sizeof(T) + 15) / 16 * 16;
  static constexpr size_t kBytes = 4 * (kL0 + kLv + kPc);
};

// padded index of the level arrays: one spare row per 8, so the 8-row
// blocks of consecutive threads start on different banks
__device__ __forceinline__ int lvx(int r) { return r + (r >> 3); }

// Level-0 rows in shared memory (element type Tin); relations stored as T
// in the same 8- or 4-byte slots.
template <class Ar, class Tin>
struct AccL0 {
  using T = typename Ar::T;
  Tin* p[4];
  int r0;
  // row r, scaled and range-checked like the multi-launch path's rows
  __device__ __forceinline__ void row(int r, T& av, T& bv, T& cv, T& dv, RowChk& k) const {
    Ar::template row<true>(p[0][r0 + r], p[1][r0 + r], p[2][r0 + r], p[3][r0 + r], av, bv, cv,
                           dv, k);
  }
  __device__ __forceinline__ T rel(int k, int r) const {
    return *reinterpret_cast<const T*>(&p[k][r0 + r]);
  }
  __device__ __forceinline__ void set_rel(int k, int r, T v) const {
    *reinterpret_cast<T*>(&p[k][r0 + r]) = v;
  }
  __device__ __forceinline__ void set_x(int r, T v) const { Ar::to(p[3][r0 + r], v); }
};

// Rows of an intra-CTA level (element type T, padded index).
template <class Ar>
struct AccLv {
  using T = typename Ar::T;
  T* p[4];
  int r0;
  __device__ __forceinline__ void row(int r, T& av, T& bv, T& cv, T& dv, RowChk&) const {
    const int i = lvx(r0 + r);
    av = p[0][i]; bv = p[1][i]; cv = p[2][i]; dv = p[3][i];
  }
  __device__ __forceinline__ T rel(int k, int r) const { return p[k][lvx(r0 + r)]; }
  __device__ __forceinline__ void set_rel(int k, int r, T v) const { p[k][lvx(r0 + r)] = v; }
  __device__ __forceinline__ void set_x(int r, T v) const { p[3][lvx(r0 + r)] = v; }
};

// Stage 1 on one block of L >= 2 rows: the same top-down sweep as k_stage1
// (f kept symbolic; x_1 = P - Q f - S x_{j+1} carried for the first reduced
// row), with every interior row's normalised relation (c/beta, g/beta,
// alpha/beta) written over its a, b, c.  red: the first reduced row
// (l_prev, f, l) and the last (f, l, f_next), four coefficients each.
template <class Ar, class Acc>
__device__ __forceinline__ void oc_fwd(const Acc& A, int L, typename Ar::T* red, bool& bad,
                                       RowChk& chk) {
  using T = typename Ar::T;
  T a0, b0, c0, d0;
  A.row(0, a0, b0, c0, d0, chk);
  T rbp = Ar::one(), cprev = Ar::zero(), g = Ar::zero(), al = Ar::neg(Ar::one());
  T P = Ar::zero(), Q = Ar::zero(), S = Ar::neg(Ar::one());
#pragma unroll 1
  for (int j = 1; j < L - 1; ++j) {
    T av, bv, cv, dv;
    A.row(j, av, bv, cv, dv, chk);
    const T ratio = Ar::mul(av, rbp);
    const T beta = Ar::sub_mul_dom(bv, ratio, cprev);
    g = Ar::sub_mul(dv, ratio, g);
    al = Ar::neg(Ar::mul(ratio, al));
    bad |= Ar::bad_pivot(beta);
    const T rbeta = Ar::rcp(beta);
    const T tt = Ar::mul(S, rbeta);
    P = Ar::sub_mul(P, tt, g);
    Q = Ar::sub_mul(Q, tt, al);
    S = Ar::neg(Ar::mul(tt, cv));
    A.set_rel(0, j, Ar::mul(cv, rbeta));
    A.set_rel(1, j, Ar::mul(g, rbeta));
    A.set_rel(2, j, Ar::mul(al, rbeta));
    rbp = rbeta;
    cprev = cv;
  }
  T av, bv, cv, dv;
  A.row(L - 1, av, bv, cv, dv, chk);
  const T ratio = Ar::mul(av, rbp);
  const T beta = Ar::sub_mul_dom(bv, ratio, cprev);
  g = Ar::sub_mul(dv, ratio, g);
  al = Ar::neg(Ar::mul(ratio, al));
  bad |= Ar::bad_pivot(beta);
  red[0] = a0;
  red[1] = Ar::sub_mul(b0, c0, Q);
  red[2] = Ar::neg(Ar::mul(c0, S));
  red[3] = Ar::sub_mul(d0, c0, P);
  red[4] = al;
  red[5] = beta;
  red[6] = cv;
  red[7] = g;
}

// Stage 3 on one block: x_0 = f, x_{L-1} = l, interior rows bottom-up from
// the stored relations; x goes to the d slots.
template <class Ar, class Acc>
__device__ __forceinline__ void oc_bwd(const Acc& A, int L, typename Ar::T f,
                                       typename Ar::T l) {
  using T = typename Ar::T;
  A.set_x(L - 1, l);
  T xn = l;
#pragma unroll 1
  for (int j = L - 2; j >= 1; --j) {
    const T cp = A.rel(0, j), gp = A.rel(1, j), ap = A.rel(2, j);
    xn = Ar::sub_mul(Ar::sub_mul(gp, ap, f), cp, xn);
    A.set_x(j, xn);
  }
  A.set_x(0, f);
}

// The intra-CTA levels of a CTA whose level-1 system (N rows, starting at
// level row 0) sits in lv: Stage 1 in kOcBlock-row blocks until at most
// kOcFinal rows are left, recording each level's offset and size; on return
// `off` and `N` describe the last level (one block).  Needs every thread.
struct OcLevels {
  int off = 0, N = 0, nl = 0;
  int offs[4], Ns[4];  // at most 3 levels: 512 -> 128 -> 32 -> 8 rows
};
template <class Ar>
__device__ __forceinline__ void oc_reduce_levels(typename Ar::T* const* lv, int N1, int tid,
                                                 OcLevels& L, bool& bad) {
  using T = typename Ar::T;
  T red[8];
  RowChk nochk;  // the level rows are computed pairs, not inputs
  L.off = 0;
  L.N = N1;
  L.nl = 0;
  while (L.N > kOcFinal) {
    const int pl = (L.N + kOcBlock - 1) / kOcBlock;
    const int noff = L.off + L.N;
    if (tid < pl) {
      const int len = tid == pl - 1 ? L.N - kOcBlock * (pl - 1) : kOcBlock;
      const AccLv<Ar> A{{lv[0], lv[1], lv[2], lv[3]}, L.off + kOcBlock * tid};
      oc_fwd<Ar>(A, len, red, bad, nochk);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        lv[q][lvx(noff + 2 * tid)] = red[q];
        lv[q][lvx(noff + 2 * tid + 1)] = red[4 + q];
      }
    }
    __syncthreads();
    L.offs[L.nl] = L.off;
    L.Ns[L.nl] = L.N;
    ++L.nl;
    L.off = noff;
    L.N = 2 * pl;
  }
}

// Stage 3 back down the levels recorded by oc_reduce_levels, given the last
// level's solution in its d slots; leaves level 1's solution in lv[3].
template <class Ar>
__device__ __forceinline__ void oc_expand_levels(typename Ar::T* const* lv, int tid,
                                                 const OcLevels& L) {
  using T = typename Ar::T;
  for (int li = L.nl - 1; li >= 0; --li) {
    const int Nl = L.Ns[li], ol = L.offs[li], pl = (Nl + kOcBlock - 1) / kOcBlock;
    const int onext = ol + Nl;
    if (tid < pl) {
      const int len = tid == pl - 1 ? Nl - kOcBlock * (pl - 1) : kOcBlock;
      const T fl = lv[3][lvx(onext + 2 * tid)], ll = lv[3][lvx(onext + 2 * tid + 1)];
      const AccLv<Ar> A{{lv[0], lv[1], lv[2], lv[3]}, ol + kOcBlock * tid};
      oc_bwd<Ar>(A, len, fl, ll);
    }
    __syncthreads();
  }
}

// a value of 4 or 8 bytes read from L2, past the (non-coherent) L1
template <class T>
__device__ __forceinline__ T ld_l2(const T* p) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element size");
  T r;
  if constexpr (sizeof(T) == 8) {
    const unsigned long long v = __ldcg(reinterpret_cast<const unsigned long long*>(p));
    memcpy(&r, &v, 8);
  } else {
    const unsigned v = __ldcg(reinterpret_cast<const unsigned*>(p));
    memcpy(&r, &v, 4);
  }
  return r;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// n rows, level-0 blocks of mt rows (p blocks, the last of length in
// [2, mt + 1]), G = ceil(p / kOcThreads) CTAs, all co-resident (cooperative
// launch).  xch: 4 x 2G values of T (the interface system); bar: a counter
// zeroed before the launch; the barrier waits for `arrivals` CTAs (G; more
// only to exercise the timeout).  vec16: a, b, c, d, x 16-byte aligned.
template <class Ar, class Tin>
__global__ void __launch_bounds__(kOcThreads, 1)
    k_onchip(int64_t n, int mt, int64_t p, const Tin* __restrict__ a, const Tin* __restrict__ b,
             const Tin* __restrict__ c, const Tin* __restrict__ d, Tin* __restrict__ x,
             typename Ar::T* __restrict__ xch, unsigned* __restrict__ bar, unsigned arrivals,
             int* __restrict__ status, int vec16, unsigned* __restrict__ dmax) {
  using T = typename Ar::T;
  using Lay = OcLayout<Ar, Tin>;
  static_assert(sizeof(T) <= sizeof(Tin), "relations are stored in the input slots");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tin* s0[4];
  T* lv[4];
  T* pc[4];
  for (int k = 0; k < 4; ++k) {
    s0[k] = reinterpret_cast<Tin*>(smem_raw + k * Lay::kL0);
    lv[k] = reinterpret_cast<T*>(smem_raw + 4 * Lay::kL0 + k * Lay::kLv);
    pc[k] = reinterpret_cast<T*>(smem_raw + 4 * (Lay::kL0 + Lay::kLv) + k * Lay::kPc);
  }
  const int G = (int)gridDim.x, cta = (int)blockIdx.x, tid = (int)threadIdx.x;
  const int64_t kb = (int64_t)cta * kOcThreads;
  const int64_t ke = kb + kOcThreads < p ? kb + kOcThreads : p;
  const int nb = (int)(ke - kb);
  const int64_t r0 = kb * mt;
  const int64_t r1 = ke == p ? n : ke * mt;
  const int rows = (int)(r1 - r0);

  // ---- load the CTA's rows (r0 * sizeof(Tin) is a multiple of 16)
  const Tin* const src[4] = {a, b, c, d};
  constexpr int V = 16 / (int)sizeof(Tin);
  const int nv = vec16 ? rows / V : 0;
  for (int k = 0; k < 4; ++k) {
    for (int i = tid; i < nv; i += kOcThreads) cp_async<16>(s0[k] + i * V, src[k] + r0 + i * V);
    for (int i = nv * V + tid; i < rows; i += kOcThreads)
      cp_async<sizeof(Tin)>(s0[k] + i, src[k] + r0 + i);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  // a[0] and c[n-1] are not part of the system
  if (tid == 0 && cta == 0) s0[0][0] = Tin{};
  if (tid == 0 && ke == p) s0[2][rows - 1] = Tin{};
  __syncthreads();

  // ---- Stage 1, level 0: one block per thread
  bool bad = false;
  T red[8];
  int L0len = 0;
  RowChk chk;
  if (tid < nb) {
    const int64_t k = kb + tid;
    L0len = k == p - 1 ? (int)(n - k * mt) : mt;
    const AccL0<Ar, Tin> A{{s0[0], s0[1], s0[2], s0[3]}, (int)(k * mt - r0)};
    oc_fwd<Ar>(A, L0len, red, bad, chk);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      lv[q][lvx(2 * tid)] = red[q];
      lv[q][lvx(2 * tid + 1)] = red[4 + q];
    }
  }
  __syncthreads();

  // the rows' range: the system's range codes (one set of atomics per
  // warp), a, c, d too large or b invalid
  if (dmax) codes_raise_warp(dmax, 0, true, chk);
  if (chk.range_bad()) atomicOr(status, ST_RANGE);
  bad |= chk.b_bad();

  // ---- Stage 1, levels 1..: 8-row blocks until one block is left
  OcLevels lev;
  oc_reduce_levels<Ar>(lv, 2 * nb, tid, lev, bad);
  const int off = lev.off, N = lev.N;
  // the CTA's own two interface equations
  const int M = 2 * G;
  if (tid == 0) {
    const AccLv<Ar> A{{lv[0], lv[1], lv[2], lv[3]}, off};
    RowChk nochk;
    oc_fwd<Ar>(A, N, red, bad, nochk);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      xch[q * M + 2 * cta] = red[q];
      xch[q * M + 2 * cta + 1] = red[4 + q];
    }
  }
  if (bad) atomicOr(status, ST_BAD_PIVOT);

  // ---- grid barrier (every CTA is resident: cooperative launch)
  __shared__ int ok_s;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    unsigned it = 0;
    while (ld_acquire_u32(bar) < arrivals) {
      if (++it > kOcSpinLimit) {
        ok = 0;
        atomicOr(status, ST_TIMEOUT);
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  if (!ok_s) return;
  // every CTA's codes are in: judge the system's range
  if (dmax && cta == 0 && tid == 0) {
    if (range_codes_bad(ld_l2(dmax), ld_l2(dmax + 1), ld_l2(dmax + 2)))
      atomicOr(status, ST_RANGE);
    dmax[0] = dmax[1] = dmax[2] = 0u;  // zero again for the next solve
  }

  // ---- Stage 2: the 2G interface rows by parallel cyclic reduction
  for (int i = tid; i < M; i += kOcThreads) {
#pragma unroll
    for (int q = 0; q < 4; ++q) pc[q][i] = ld_l2(xch + q * M + i);
  }
  __syncthreads();
  constexpr int kPer = (2 * kOcMaxCtas + kOcThreads - 1) / kOcThreads;
  bool badr = false;
  for (int s = 1; s < M; s <<= 1) {
    T na[kPer], nbv[kPer], nc[kPer], nd[kPer];
#pragma unroll
    for (int h = 0; h < kPer; ++h) {
      const int i = tid + kOcThreads * h;
      if (i < M) {
        const int im = i - s, ip = i + s;
        const T am = im >= 0 ? pc[0][im] : Ar::zero(), bm = im >= 0 ? pc[1][im] : Ar::one();
        const T cm = im >= 0 ? pc[2][im] : Ar::zero(), dm = im >= 0 ? pc[3][im] : Ar::zero();
        const T ap = ip < M ? pc[0][ip] : Ar::zero(), bp = ip < M ? pc[1][ip] : Ar::one();
        const T cp = ip < M ? pc[2][ip] : Ar::zero(), dp = ip < M ? pc[3][ip] : Ar::zero();
        badr |= Ar::bad_pivot(bm) | Ar::bad_pivot(bp);
        const T k1 = Ar::mul(pc[0][i], Ar::rcp(bm));
        const T k2 = Ar::mul(pc[2][i], Ar::rcp(bp));
        na[h] = Ar::neg(Ar::mul(am, k1));
        nc[h] = Ar::neg(Ar::mul(cp, k2));
        nbv[h] = Ar::sub_mul(Ar::sub_mul(pc[1][i], cm, k1), ap, k2);
        nd[h] = Ar::sub_mul(Ar::sub_mul(pc[3][i], dm, k1), dp, k2);
      }
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < kPer; ++h) {
      const int i = tid + kOcThreads * h;
      if (i < M) {
        pc[0][i] = na[h];
        pc[1][i] = nbv[h];
        pc[2][i] = nc[h];
        pc[3][i] = nd[h];
      }
    }
    __syncthreads();
  }
  if (badr && cta == 0) atomicOr(status, ST_BAD_PIVOT);
  const T fc = Ar::mul(pc[3][2 * cta], Ar::rcp(pc[1][2 * cta]));
  const T lc = Ar::mul(pc[3][2 * cta + 1], Ar::rcp(pc[1][2 * cta + 1]));

  // ---- Stage 3 down the levels
  if (tid == 0) {
    const AccLv<Ar> A{{lv[0], lv[1], lv[2], lv[3]}, off};
    oc_bwd<Ar>(A, N, fc, lc);
  }
  __syncthreads();
  oc_expand_levels<Ar>(lv, tid, lev);
  if (tid < nb) {
    const int64_t k = kb + tid;
    const T fl = lv[3][lvx(2 * tid)], ll = lv[3][lvx(2 * tid + 1)];
    const AccL0<Ar, Tin> A{{s0[0], s0[1], s0[2], s0[3]}, (int)(k * mt - r0)};
    oc_bwd<Ar>(A, L0len, fl, ll);
  }
  __syncthreads();

  // ---- x out of the d slots
  for (int i = tid; i < nv; i += kOcThreads)
    *reinterpret_cast<float4*>(x + r0 + i * V) = *reinterpret_cast<const float4*>(s0[3] + i * V);
  for (int i = nv * V + tid; i < rows; i += kOcThreads) x[r0 + i] = s0[3][i];
  bool oob = false;
  for (int i = tid; i < rows; i += kOcThreads) oob |= Ar::out_bad(s0[3][i]);
  if (oob) atomicOr(status, ST_RANGE);
}

}  // namespace tps

namespace tps {

// ------------------------------------------------------------------ truncated decoupling
// Not the paper's method: an approximation for strongly dominant systems
// (TPS_TRUNCATE).  Window w keeps rows [wR, wR + R) and is solved, on chip
// in one CTA, as the tridiagonal system on the extended rows
// [wR - h, wR + R + h) (clipped to [0, n)) with the couplings that leave that
// range cut.  With q = max (|a| + |c|) / |b| over the window (cut couplings
// zero) the inverse of the window's matrix decays like q^|i-j|, so the kept
// rows differ from the exact solution by at most
//     (|a_cut| q^dl + |c_cut| q^dr) / ((1 - q) min |b|) * ||x||_inf,
// dl, dr the distances from the kept rows to the two cut ends.  Each window
// publishes that bound (maximum over windows, as the bits of a
// non-negative float) and flags ST_NO_CONVERGENCE where it exceeds `tol`.
constexpr int kWinThreads = 128;
constexpr int kWinRowsMax = 1792;              // extended rows of one window
constexpr int kWinLevelRows = 256 + 64 + 16 + 4;
constexpr int kWinLevelSlots = kWinLevelRows + kWinLevelRows / kOcBlock + kOcBlock;

// Shared memory of a window of at most `rows` extended rows: the level
// arrays first (fixed size), then four row arrays of `rows` elements.
template <class Ar, class Tin>
struct WinLayout {
  using T = typename Ar::T;
  static constexpr size_t kLv = ((size_t)kWinLevelSlots * sizeof(T) + 15) / 16 * 16;
  __host__ __device__ static constexpr size_t l0(int rows) {
    return ((size_t)rows * sizeof(Tin) + 15) / 16 * 16;
  }
  __host__ __device__ static constexpr size_t bytes(int rows) { return 4 * (kLv + l0(rows)); }
};


// R, h even; one CTA per window.
template <class Ar, class Tin>
__global__ void __launch_bounds__(kWinThreads)
    k_window(int64_t n, int R, int h, const Tin* __restrict__ a, const Tin* __restrict__ b,
             const Tin* __restrict__ c, const Tin* __restrict__ d, Tin* __restrict__ x, float tol,
             unsigned* __restrict__ bound_max, int* __restrict__ status, int vec16,
             unsigned* __restrict__ dmax) {
  using T = typename Ar::T;
  using Lay = WinLayout<Ar, Tin>;
  static_assert(sizeof(T) <= sizeof(Tin), "relations are stored in the input slots");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tin* s0[4];
  T* lv[4];
  const size_t l0 = Lay::l0(R + 2 * h);
  for (int k = 0; k < 4; ++k) {
    lv[k] = reinterpret_cast<T*>(smem_raw + k * Lay::kLv);
    s0[k] = reinterpret_cast<Tin*>(smem_raw + 4 * Lay::kLv + k * l0);
  }
  __shared__ unsigned q_bits, bmin_key;
  __shared__ Tin cut_s[2];
  const int tid = (int)threadIdx.x;
  const int64_t k0 = (int64_t)blockIdx.x * R;
  const int64_t k1 = k0 + R < n ? k0 + R : n;
  const int64_t e0 = k0 - h > 0 ? k0 - h : 0;
  const int64_t e1 = k1 + h < n ? k1 + h : n;
  const int E = (int)(e1 - e0);

  // ---- load the extended rows (16-byte pieces only where the window start
  // is a whole number of pieces from the 16-byte aligned base)
  const Tin* const src[4] = {a, b, c, d};
  constexpr int V = 16 / (int)sizeof(Tin);
  const int nv = (vec16 && e0 % V == 0) ? E / V : 0;
  for (int k = 0; k < 4; ++k) {
    for (int i = tid; i < nv; i += kWinThreads) cp_async<16>(s0[k] + i * V, src[k] + e0 + i * V);
    for (int i = nv * V + tid; i < E; i += kWinThreads)
      cp_async<sizeof(Tin)>(s0[k] + i, src[k] + e0 + i);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();  // every thread's copies have landed
  if (tid == 0) {
    cut_s[0] = e0 > 0 ? s0[0][0] : Tin{};  // the couplings being cut
    cut_s[1] = e1 < n ? s0[2][E - 1] : Tin{};
    q_bits = 0u;
    bmin_key = 0x7FFFFFFFu;
    s0[0][0] = Tin{};
    s0[2][E - 1] = Tin{};
  }
  __syncthreads();
  // ---- q and min |b| of the window (cut couplings zero): q per row from
  // the scaled row, rounded up; min |b| as the smallest magnitude key
  float qmax = 0.0f;
  unsigned bkey = 0x7FFFFFFFu;
  for (int i = tid; i < E; i += kWinThreads) {
    qmax = fmaxf(qmax, win_row_q(s0[0][i], s0[1][i], s0[2][i]));
    bkey = min(bkey, mag_key(s0[1][i]));
  }
  // truncated parts and fp32 rounding: widen q by a relative 2^-20 margin
  qmax = __fmul_ru(qmax, 1.0f + 9.5367431640625e-07f);
  atomicMax(&q_bits, __float_as_uint(qmax));
  atomicMin(&bmin_key, bkey);
  __syncthreads();  // every row read before Stage 1 overwrites a, b, c in place

  // ---- Stage 1: thread blocks of mt rows (odd) over the E rows, then levels
  int mt = (E + kWinThreads - 1) / kWinThreads;
  if (mt < 3) mt = 3;
  mt |= 1;
  int p = (E + mt - 1) / mt;
  if (p > 1 && E - (p - 1) * mt == 1) --p;  // merge a one-row tail
  bool bad = false;
  T red[8];
  RowChk chk;
  const int myL = tid < p ? (tid == p - 1 ? E - tid * mt : mt) : 0;
  if (tid < p) {
    const AccL0<Ar, Tin> A{{s0[0], s0[1], s0[2], s0[3]}, tid * mt};
    oc_fwd<Ar>(A, myL, red, bad, chk);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      lv[q][lvx(2 * tid)] = red[q];
      lv[q][lvx(2 * tid + 1)] = red[4 + q];
    }
  }
  __syncthreads();
  // the rows' range (the system-wide |d / b| test runs after the launch)
  if (dmax) codes_raise_warp(dmax, 0, true, chk);
  if (chk.range_bad()) atomicOr(status, ST_RANGE);
  bad |= chk.b_bad();
  OcLevels lev;
  oc_reduce_levels<Ar>(lv, 2 * p, tid, lev, bad);
  // ---- the window's two interface equations, with nothing outside: a 2x2 system
  if (tid == 0) {
    const AccLv<Ar> A{{lv[0], lv[1], lv[2], lv[3]}, lev.off};
    RowChk nochk;
    oc_fwd<Ar>(A, lev.N, red, bad, nochk);
    // b1 f + c1 l = d1;  a2 f + b2 l = d2, eliminated as two Thomas rows:
    // no product of two pivots is formed (native fp64 rows of any scale,
    // e.g. 2^-600, whose determinant would underflow)
    bad |= Ar::bad_pivot(red[1]);
    const T r1 = Ar::rcp(red[1]);
    const T g1 = Ar::mul(red[2], r1);  // c1 / b1
    const T z1 = Ar::mul(red[3], r1);  // d1 / b1
    const T b2p = Ar::sub_mul(red[5], red[4], g1);
    bad |= Ar::bad_pivot(b2p);
    const T l = Ar::mul(Ar::sub_mul(red[7], red[4], z1), Ar::rcp(b2p));
    const T f = Ar::sub_mul(z1, g1, l);
    oc_bwd<Ar>(A, lev.N, f, l);
  }
  __syncthreads();
  oc_expand_levels<Ar>(lv, tid, lev);
  if (tid < p) {
    const T fl = lv[3][lvx(2 * tid)], ll = lv[3][lvx(2 * tid + 1)];
    const AccL0<Ar, Tin> A{{s0[0], s0[1], s0[2], s0[3]}, tid * mt};
    oc_bwd<Ar>(A, myL, fl, ll);
  }
  if (bad) atomicOr(status, ST_BAD_PIVOT);
  __syncthreads();

  // ---- the kept rows out (16-byte pieces where both the global row k0 and
  // the shared-memory row o are whole pieces from aligned bases)
  const int o = (int)(k0 - e0), K = (int)(k1 - k0);
  const int kv = (vec16 && k0 % V == 0 && o % V == 0) ? K / V : 0;
  for (int i = tid; i < kv; i += kWinThreads)
    *reinterpret_cast<float4*>(x + k0 + i * V) =
        *reinterpret_cast<const float4*>(s0[3] + o + i * V);
  for (int i = kv * V + tid; i < K; i += kWinThreads) x[k0 + i] = s0[3][o + i];
  bool oob = false;
  for (int i = tid; i < K; i += kWinThreads) oob |= Ar::out_bad(s0[3][o + i]);
  if (oob) atomicOr(status, ST_RANGE);

  // ---- the window's truncation bound
  if (tid == 0) {
    const float q = __uint_as_float(q_bits);
    // |a_cut| / min |b| and |c_cut| / min |b|, rounded up (scale-free, so a
    // system scaled anywhere in the input's range gets the same bound)
    float ra, rc;
    if constexpr (sizeof(Tin) == 8) {
      const double bmd = __hiloint2double((int)bmin_key, 0);
      ra = __double2float_ru(__ddiv_ru(fabs((double)cut_s[0]), bmd));
      rc = __double2float_ru(__ddiv_ru(fabs((double)cut_s[1]), bmd));
    } else {
      const float bmf = __uint_as_float(bmin_key);
      ra = __fdiv_ru(fabsf((float)cut_s[0]), bmf);
      rc = __fdiv_ru(fabsf((float)cut_s[1]), bmf);
    }
    float eps;
    if (ra == 0.0f && rc == 0.0f) {
      eps = 0.0f;  // nothing cut
    } else if (!(q < 1.0f) || !(ra < __int_as_float(0x7f800000)) ||
               !(rc < __int_as_float(0x7f800000))) {
      eps = __int_as_float(0x7f800000);
    } else {
      const float num = __fadd_ru(__fmul_ru(ra, powf(q, (float)o)),
                                  __fmul_ru(rc, powf(q, (float)(e1 - k1))));
      eps = __fdiv_ru(num, __fsub_rd(1.0f, q)) * (1.0f + 1e-5f);
    }
    atomicMax(bound_max, __float_as_uint(eps));
    if (!(eps <= tol)) atomicOr(status, ST_NO_CONVERGENCE);
  }
}

}  // namespace tps
