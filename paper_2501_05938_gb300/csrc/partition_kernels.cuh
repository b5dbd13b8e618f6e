// Stage 1, Stage 3 and the small-system solve of the tridiagonal partition
// method (Sec. 1 and Sec. 2.2 of the paper: per-block elimination onto the
// interface unknowns, a reduced interface solve, per-block recovery).
//
// System: a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i]; a[0], c[n-1] unused.
// Blocks: block k owns rows k*m .. k*m + L_k - 1, L_k = m except the last
// block, whose length Llast lies in [2, m + 1] (a one-row tail is merged into
// the block before it).  The first and last row of each block are its
// interface unknowns f_k and l_k; the reduced system in (f_0, l_0, f_1, ...)
// is tridiagonal, so row 2k is block k's "first" equation in
// (l_{k-1}, f_k, l_k) and row 2k+1 its "last" equation in (f_k, l_k, f_{k+1}).
//
// GPU mapping.  One lane owns one block and sweeps it serially (the
// recurrences are first-order); a warp owns 32 consecutive blocks.  The warp
// streams its blocks in chunks of R rows: for each of a, b, c, d it copies
// 32 blocks x R rows into shared memory with cp.async (each block's R rows
// are contiguous in global memory, so the copies coalesce), double
// buffered, with a padded stride of R+1 elements per block so that lane j
// reading row r of block j hits distinct banks.
//
// Stage 1 is a single top-down sweep per block.  Writing the interior
// relation after row j as  beta_j x_j + c_j x_{j+1} = g_j - alpha_j f  (a
// forward elimination that keeps f symbolic), the last reduced equation is
// the relation after the block's last row, (alpha, beta, c, g) on
// (f_k, l_k, f_{k+1}).  The first reduced equation needs the first interior
// unknown as a function of f_k and l_k; instead of a second, bottom-up
// sweep, the sweep carries x_1 = P - Q f - S x_{j+1} along, which costs four
// multiply-adds per row and no extra reciprocal.  Every K = R rows the
// normalised relation x_j = (g_j - alpha_j f - c_j x_{j+1}) / beta_j is
// written out as a checkpoint (c/beta, g/beta, alpha/beta).
//
// Stage 3 walks each block's chunks bottom-up.  A chunk restarts the forward
// elimination from its checkpoint (with f now known), keeps the R pivots and
// right-hand sides in registers, and back-substitutes from the x of the row
// below it (l_k for the last chunk).  The result goes through the chunk's
// shared-memory slots so the stores coalesce like the loads.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "arith.cuh"

namespace tps {

// ------------------------------------------------------------------ cp.async
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (BYTES == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
  } else {
    static_assert(BYTES == 4, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------------------ geometry
struct Level {
  int64_t n;        // rows
  int64_t p;        // blocks
  int64_t k_begin;  // blocks this launch processes: [k_begin, k_end)
  int64_t k_end;
  int32_t m;        // nominal block length
  int32_t llast;    // length of block p-1, in [2, m+1]
  int32_t ncap;     // checkpoint slots per block
  int32_t pad;
};

__device__ __forceinline__ int block_len(const Level& lv, int64_t k) {
  return k == lv.p - 1 ? lv.llast : lv.m;
}

// Status bits written into the device status word.
enum : int { ST_BAD_PIVOT = 1, ST_NO_CONVERGENCE = 2, ST_TIMEOUT = 4 };

template <class Tin, int R>
struct WarpTile {
  static constexpr int kStride = R + 1;                 // padded row stride per block
  static constexpr int kArr = 32 * kStride;             // one array of the chunk
  static constexpr int kBuf = 4 * kArr;                 // a, b, c, d
  static constexpr int kWarp = 2 * kBuf;                // double buffered
  static constexpr size_t kBytesPerWarp = sizeof(Tin) * kWarp;
};

// Copy rows [row0, row0 + R) of the warp's blocks (clipped to each block's
// length) of the four arrays into one buffer.  Lane l copies elements
// e = l + 32 j, e -> (block e / R, row e % R), so consecutive lanes read
// consecutive rows of one block.
template <class Tin, int R>
__device__ __forceinline__ void load_chunk(Tin* buf, const Tin* __restrict__ a,
                                           const Tin* __restrict__ b, const Tin* __restrict__ c,
                                           const Tin* __restrict__ d, const Level& lv, int64_t k0,
                                           int nb, int row0, int lane) {
  using WT = WarpTile<Tin, R>;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int e = lane + 32 * j;
    const int blk = e / R;
    const int r = e % R;
    const int row = row0 + r;
    if (blk < nb && row < block_len(lv, k0 + blk)) {
      const int64_t g = (k0 + blk) * (int64_t)lv.m + row;
      const int s = blk * WT::kStride + r;
      cp_async<sizeof(Tin)>(buf + 0 * WT::kArr + s, a + g);
      cp_async<sizeof(Tin)>(buf + 1 * WT::kArr + s, b + g);
      cp_async<sizeof(Tin)>(buf + 2 * WT::kArr + s, c + g);
      cp_async<sizeof(Tin)>(buf + 3 * WT::kArr + s, d + g);
    }
  }
}

__device__ __forceinline__ int warp_chunks(const Level& lv, int64_t k0, int nb, int R) {
  // only the warp holding block p-1 can have a block longer than m
  const int lmax = (k0 + nb == lv.p) ? max(lv.m, lv.llast) : lv.m;
  return (lmax + R - 1) / R;
}

// ------------------------------------------------------------------ Stage 1
template <class Ar, class Tin, class Tred, int R, int W>
__global__ void __launch_bounds__(W * 32)
    k_stage1(Level lv, const Tin* __restrict__ a, const Tin* __restrict__ b,
             const Tin* __restrict__ c, const Tin* __restrict__ d, Tred* __restrict__ ra,
             Tred* __restrict__ rb, Tred* __restrict__ rc, Tred* __restrict__ rd,
             Tred* __restrict__ ck_gam, Tred* __restrict__ ck_y, Tred* __restrict__ ck_v,
             int* __restrict__ status) {
  using T = typename Ar::T;
  using WT = WarpTile<Tin, R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k0 = lv.k_begin + ((int64_t)blockIdx.x * W + warp) * 32;
  if (k0 >= lv.k_end) return;
  const int nb = (int)(lv.k_end - k0 < 32 ? lv.k_end - k0 : 32);
  Tin* tile = reinterpret_cast<Tin*>(smem_raw) + warp * WT::kWarp;
  const int64_t k = k0 + lane;
  const bool active = lane < nb;
  const int L = active ? block_len(lv, k) : 0;
  const int nch = warp_chunks(lv, k0, nb, R);

  // virtual state before row 1 (relation x_0 = f): rbeta = 1, c_prev = 0,
  // g = 0, alpha = -1; first interior unknown x_1 = P - Q f - S x_1 with
  // P = Q = 0, S = -1.
  T rbp = Ar::one(), cprev = Ar::zero(), g = Ar::zero(), al = Ar::neg(Ar::one());
  T P = Ar::zero(), Q = Ar::zero(), S = Ar::neg(Ar::one());
  T a0 = Ar::zero(), b0 = Ar::one(), c0 = Ar::zero(), d0 = Ar::zero();
  T beta = Ar::one(), clast = Ar::zero();
  bool bad = false;

  load_chunk<Tin, R>(tile, a, b, c, d, lv, k0, nb, 0, lane);
  cp_async_commit();
  for (int ch = 0; ch < nch; ++ch) {
    if (ch + 1 < nch)
      load_chunk<Tin, R>(tile + ((ch + 1) & 1) * WT::kBuf, a, b, c, d, lv, k0, nb, (ch + 1) * R,
                         lane);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    const Tin* t = tile + (ch & 1) * WT::kBuf + lane * WT::kStride;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = ch * R + r;
      if (row < L) {
        const T av = Ar::from(t[0 * WT::kArr + r]);
        const T bv = Ar::from(t[1 * WT::kArr + r]);
        const T cv = Ar::from(t[2 * WT::kArr + r]);
        const T dv = Ar::from(t[3 * WT::kArr + r]);
        if (row == 0) {
          a0 = av; b0 = bv; c0 = cv; d0 = dv;
        } else {
          const T ratio = Ar::mul(av, rbp);
          beta = Ar::sub_mul(bv, ratio, cprev);
          g = Ar::sub_mul(dv, ratio, g);
          al = Ar::neg(Ar::mul(ratio, al));
          if (row < L - 1) {
            bad |= Ar::bad_pivot(beta);
            const T rbeta = Ar::rcp(beta);
            const T tt = Ar::mul(S, rbeta);
            P = Ar::sub_mul(P, tt, g);
            Q = Ar::sub_mul(Q, tt, al);
            S = Ar::neg(Ar::mul(tt, cv));
            rbp = rbeta;
            cprev = cv;
            if (((row + 1) % R) == 0 && row <= L - 3) {
              const int64_t slot = (int64_t)((row + 1) / R - 1) * lv.p + k;
              Ar::to(ck_gam[slot], Ar::mul(cv, rbeta));
              Ar::to(ck_y[slot], Ar::mul(g, rbeta));
              Ar::to(ck_v[slot], Ar::mul(al, rbeta));
            }
          } else {
            clast = cv;
          }
        }
      }
    }
    __syncwarp();
  }
  if (active) {
    bad |= Ar::bad_pivot(beta);
    // first equation of block k, unknowns (l_{k-1}, f_k, l_k)
    Ar::to(ra[2 * k], k == 0 ? Ar::zero() : a0);
    Ar::to(rb[2 * k], Ar::sub_mul(b0, c0, Q));
    Ar::to(rc[2 * k], Ar::neg(Ar::mul(c0, S)));
    Ar::to(rd[2 * k], Ar::sub_mul(d0, c0, P));
    // last equation of block k, unknowns (f_k, l_k, f_{k+1})
    Ar::to(ra[2 * k + 1], al);
    Ar::to(rb[2 * k + 1], beta);
    Ar::to(rc[2 * k + 1], k == lv.p - 1 ? Ar::zero() : clast);
    Ar::to(rd[2 * k + 1], g);
    if (bad) atomicOr(status, ST_BAD_PIVOT);
  }
}

// ------------------------------------------------------------------ Stage 3
template <class Ar, class Tin, class Tred, int R, int W>
__global__ void __launch_bounds__(W * 32)
    k_stage3(Level lv, const Tin* __restrict__ a, const Tin* __restrict__ b,
             const Tin* __restrict__ c, const Tin* __restrict__ d, const Tred* __restrict__ xred,
             const Tred* __restrict__ ck_gam, const Tred* __restrict__ ck_y,
             const Tred* __restrict__ ck_v, Tin* __restrict__ x, int* __restrict__ status) {
  using T = typename Ar::T;
  using WT = WarpTile<Tin, R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k0 = lv.k_begin + ((int64_t)blockIdx.x * W + warp) * 32;
  if (k0 >= lv.k_end) return;
  const int nb = (int)(lv.k_end - k0 < 32 ? lv.k_end - k0 : 32);
  Tin* tile = reinterpret_cast<Tin*>(smem_raw) + warp * WT::kWarp;
  const int64_t k = k0 + lane;
  const bool active = lane < nb;
  const int L = active ? block_len(lv, k) : 0;
  const int nch = warp_chunks(lv, k0, nb, R);

  T f = Ar::zero(), l = Ar::zero();
  if (active) {
    f = Ar::from(xred[2 * k]);
    l = Ar::from(xred[2 * k + 1]);
  }
  T xnext = l;  // x of the row below the chunk being processed
  bool bad = false;

  // chunks bottom-up: ch = nch-1 .. 0, buffer parity by visiting order
  load_chunk<Tin, R>(tile, a, b, c, d, lv, k0, nb, (nch - 1) * R, lane);
  cp_async_commit();
  for (int it = 0; it < nch; ++it) {
    const int ch = nch - 1 - it;
    if (ch > 0)
      load_chunk<Tin, R>(tile + ((it + 1) & 1) * WT::kBuf, a, b, c, d, lv, k0, nb, (ch - 1) * R,
                         lane);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    Tin* t = tile + (it & 1) * WT::kBuf + lane * WT::kStride;

    // relation entering the chunk: x_{row0-1} = zp - gp * x_{row0}
    T zp = f, gp = Ar::zero();
    if (active && ch > 0 && ch * R <= L - 2) {
      const int64_t slot = (int64_t)(ch - 1) * lv.p + k;
      gp = Ar::from(ck_gam[slot]);
      zp = Ar::sub_mul(Ar::from(ck_y[slot]), Ar::from(ck_v[slot]), f);
    }
    T Z[R], G[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = ch * R + r;
      Z[r] = Ar::zero();
      G[r] = Ar::zero();
      if (row >= 1 && row <= L - 2) {
        const T av = Ar::from(t[0 * WT::kArr + r]);
        const T bv = Ar::from(t[1 * WT::kArr + r]);
        const T cv = Ar::from(t[2 * WT::kArr + r]);
        const T dv = Ar::from(t[3 * WT::kArr + r]);
        const T beta = Ar::sub_mul(bv, av, gp);
        bad |= Ar::bad_pivot(beta);
        const T rbeta = Ar::rcp(beta);
        zp = Ar::mul(Ar::sub_mul(dv, av, zp), rbeta);
        gp = Ar::mul(cv, rbeta);
        Z[r] = zp;
        G[r] = gp;
      }
    }
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      const int row = ch * R + r;
      if (row < L) {
        T xr;
        if (row == L - 1) {
          xr = l;
        } else if (row == 0) {
          xr = f;
        } else {
          xr = Ar::sub_mul(Z[r], G[r], xnext);
          xnext = xr;
        }
        Ar::to(t[0 * WT::kArr + r], xr);  // a is no longer needed: reuse its slot
      }
    }
    __syncwarp();
    // coalesced write-back of the chunk's x, same element mapping as the load
    {
      const Tin* tx = tile + (it & 1) * WT::kBuf;
      const int row0 = ch * R;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int e = lane + 32 * j;
        const int blk = e / R;
        const int r = e % R;
        const int row = row0 + r;
        if (blk < nb && row < block_len(lv, k0 + blk))
          x[(k0 + blk) * (int64_t)lv.m + row] = tx[blk * WT::kStride + r];
      }
    }
    __syncwarp();
  }
  if (active && bad) atomicOr(status, ST_BAD_PIVOT);
}

// ------------------------------------------------------------------ small systems
// One warp solves a system of n <= 64 rows by parallel cyclic reduction
// (Hockney 1965): at stride s every row eliminates its neighbours at
// distance s, after ceil(log2 n) steps each row is decoupled and
// x_i = d_i / b_i.  Rows outside [0, n) act as identity rows.
constexpr int kBaseMax = 64;

template <class Ar, class Tin, class Tout>
__global__ void __launch_bounds__(32)
    k_base(int64_t n, const Tin* __restrict__ a, const Tin* __restrict__ b,
           const Tin* __restrict__ c, const Tin* __restrict__ d, Tout* __restrict__ x,
           int* __restrict__ status) {
  using T = typename Ar::T;
  __shared__ T sa[kBaseMax], sb[kBaseMax], sc[kBaseMax], sd[kBaseMax];
  const int lane = threadIdx.x;
  const int nn = (int)n;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    if (i < nn) {
      sa[i] = (i == 0) ? Ar::zero() : Ar::from(a[i]);
      sb[i] = Ar::from(b[i]);
      sc[i] = (i == nn - 1) ? Ar::zero() : Ar::from(c[i]);
      sd[i] = Ar::from(d[i]);
    } else {
      sa[i] = Ar::zero(); sb[i] = Ar::one(); sc[i] = Ar::zero(); sd[i] = Ar::zero();
    }
  }
  __syncwarp();
  bool bad = false;
  for (int s = 1; s < nn; s <<= 1) {
    T na[2], nbv[2], nc[2], nd[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      const int im = i - s, ip = i + s;
      const T am = im >= 0 ? sa[im] : Ar::zero();
      const T bm = im >= 0 ? sb[im] : Ar::one();
      const T cm = im >= 0 ? sc[im] : Ar::zero();
      const T dm = im >= 0 ? sd[im] : Ar::zero();
      const T ap = ip < kBaseMax ? sa[ip] : Ar::zero();
      const T bp = ip < kBaseMax ? sb[ip] : Ar::one();
      const T cp = ip < kBaseMax ? sc[ip] : Ar::zero();
      const T dp = ip < kBaseMax ? sd[ip] : Ar::zero();
      bad |= Ar::bad_pivot(bm) | Ar::bad_pivot(bp);
      const T k1 = Ar::mul(sa[i], Ar::rcp(bm));
      const T k2 = Ar::mul(sc[i], Ar::rcp(bp));
      na[h] = Ar::neg(Ar::mul(am, k1));
      nc[h] = Ar::neg(Ar::mul(cp, k2));
      nbv[h] = Ar::sub_mul(Ar::sub_mul(sb[i], cm, k1), ap, k2);
      nd[h] = Ar::sub_mul(Ar::sub_mul(sd[i], dm, k1), dp, k2);
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      sa[i] = na[h]; sb[i] = nbv[h]; sc[i] = nc[h]; sd[i] = nd[h];
    }
    __syncwarp();
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    if (i < nn) {
      bad |= Ar::bad_pivot(sb[i]);
      Ar::to(x[i], Ar::mul(sd[i], Ar::rcp(sb[i])));
    }
  }
  if (bad) atomicOr(status, ST_BAD_PIVOT);
}

}  // namespace tps
