// Truncated decoupling (TPS_TRUNCATE) as one warp per window, one pass over
// HBM.  Not a method of the paper: an approximation for strongly dominant
// systems that drops the couplings beyond a halo of h rows around each
// window of R kept rows, so every window is solved on its own (the
// definition and error bound are those of the truncation oracle).
//
// Window w keeps rows [w R, w R + R) and is solved on its extended rows
// [w R - h, w R + R + h) (clipped to [0, n)), 32 mb rows for R + 2 h = 32 mb.
// The extended rows split into 32 blocks of mb rows, one per lane; the
// partition method (Sec. 1 and Sec. 2.2 of the paper) then runs inside the
// warp:
//   Stage 1  every lane sweeps its block top-down (16-byte cp.async tiles of
//            8-row chunks, as the level-0 kernels), in a divided form whose
//            per-row quantities are the interior row's relation
//                x_j = g'_j - alpha'_j f - c'_j x_{j+1},
//            (c'_j, g'_j, alpha'_j) = (c_j, g_j, alpha_j) / beta_j, written to
//            the window's slice of a relation buffer (read back once and then
//            discarded from L2; what L2 still holds at that point never goes
//            to DRAM, at the default window size about a third), and forms
//            the block's two reduced rows;
//   Stage 2  the window's 64 reduced rows, with the couplings that leave the
//            extended range cut, by parallel cyclic reduction in the warp;
//   Stage 3  every lane walks its block bottom-up through the relations
//            (staged in shared memory by cp.async) and writes the rows it
//            keeps through the same coalesced tiles.
// a, b, c, d are read from HBM once (the halo rows twice: they are kept rows
// of the neighbouring windows), x written once.  The window's error bound
//     (|a_cut| q^dl + |c_cut| q^dr) / ((1 - q) min |b|)  (relative to max |x|)
// with q = max (|a| + |c|) / |b| over its extended rows (cut couplings 0) is
// published as the bits of a non-negative float (atomicMax); a window above
// `tol` sets ST_NO_CONVERGENCE.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "partition_kernels.cuh"
#include "window_bound.cuh"

namespace tps {

constexpr int kWinBlockMin = 8;    // rows per lane block, bounds of the warp windows
constexpr int kWinBlockMax = 256;
constexpr int kWinChunk = 8;       // Stage-1 chunk rows (all element types)

// Geometry of a warp window.  B[l] .. B[l+1] is lane l's block (rows of the
// system), l = 0 .. 31; a block of one row (a clip at 0 or n) is merged
// into its neighbour, so every non-empty block has at least two rows.
struct WinGeom {
  int64_t e0, e1;  // extended rows [e0, e1) (clipped)
  int64_t k0, k1;  // kept rows [k0, k1)
  __device__ __forceinline__ void init(int64_t n, int R, int h, int64_t w) {
    k0 = w * (int64_t)R;
    k1 = k0 + R < n ? k0 + R : n;
    e0 = k0 - h > 0 ? k0 - h : 0;
    e1 = k1 + h < n ? k1 + h : n;
  }
  // Lane l's block [b0, b1) for block rows mb: the boundaries o + l mb
  // (o = k0 - h) clipped to [e0, e1].  A clip can leave a one-row block at
  // either end; that row goes to the neighbouring block (which then has up
  // to mb + 2 rows), so every non-empty block has at least two rows.
  __device__ __forceinline__ void block(int mb, int h, int l, int64_t& b0, int64_t& b1) const {
    const int64_t o = k0 - h;
    auto C = [&](int j) {
      const int64_t v = o + (int64_t)j * mb;
      return v < e0 ? e0 : (v > e1 ? e1 : v);
    };
    const int64_t cm = C(l - 1), c0 = C(l), c1 = C(l + 1), c2 = C(l + 2);
    b0 = c0;
    b1 = c1;
    if (c0 == e0 && c1 == e0 + 1) b1 = c0;  // give the first one-row block away
    if (cm == e0 && c0 == e0 + 1) b0 = e0;  // ... to this lane
    if (c0 == e1 - 1 && c1 == e1) b0 = e1;  // give the last one-row block away
    if (c1 == e1 - 1 && c2 == e1) b1 = e1;  // ... to this lane
    if (b1 < b0) b1 = b0;
  }
};

}  // namespace tps

namespace tps {

// The 16-byte pieces lane `lane` copies for every array of a window's
// chunk: piece q = lane + 32 j is piece q % kPieces of block q / kPieces
// (the same mapping as the level-0 kernels' PieceMap).
template <class Tin, int R>
struct WinPieces {
  using TL = Tile<Tin, R>;
  int64_t goff[TL::kPieces];  // element offset of the piece in the arrays (chunk 0)
  int soff[TL::kPieces];      // element offset in a buffer's array
  int row[TL::kPieces];       // first row of the piece within its block (chunk 0)
  int len[TL::kPieces];       // length of the piece's block (0: empty)
  __device__ __forceinline__ void init(const WinGeom& G, int mb, int h, int lane) {
#pragma unroll
    for (int j = 0; j < TL::kPieces; ++j) {
      const int q = lane + 32 * j;
      const int blk = q / TL::kPieces;
      const int pc = q % TL::kPieces;
      int64_t s0, s1;
      G.block(mb, h, blk, s0, s1);
      row[j] = pc * TL::kVec;
      len[j] = (int)(s1 - s0);
      goff[j] = s0 + row[j];
      soff[j] = blk * TL::kStride + row[j];
    }
  }
};

// Write the kept rows [k0, k1) among rows [row0, row0 + R) of the warp's
// blocks from the buffer's first array to x.
template <class Tin, int R, bool kVec16>
__device__ __forceinline__ void store_kept(Tin* __restrict__ x, const Tin* buf,
                                           const WinPieces<Tin, R>& pm, int row0, int64_t k0,
                                           int64_t k1) {
  using TL = Tile<Tin, R>;
#pragma unroll
  for (int j = 0; j < TL::kPieces; ++j) {
    const int avail = pm.len[j] - (row0 + pm.row[j]);
    const int64_t g = pm.goff[j] + row0;
    if (kVec16 && avail >= TL::kVec && g >= k0 && g + TL::kVec <= k1) {
      *reinterpret_cast<float4*>(x + g) = *reinterpret_cast<const float4*>(buf + pm.soff[j]);
    } else if (avail > 0) {
#pragma unroll
      for (int v = 0; v < TL::kVec; ++v)
        if (v < avail && g + v >= k0 && g + v < k1) x[g + v] = buf[pm.soff[j] + v];
    }
  }
}

// A value's leading binary32 part, for the window's dominance factor: the
// high part of a pair, or the value rounded (native fp64: a conversion
// instruction of the slow fp64 pipe; that path is bound by the pipe anyway).
__device__ __forceinline__ float lead_f32(const df64& v) { return v.hi; }
__device__ __forceinline__ float lead_f32(float v) { return v; }

__device__ __forceinline__ void discard_l2(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(p) : "memory");
}

// Rows of one window's relation slice (block rows up to mb + 2, whole chunks).
__host__ __device__ __forceinline__ int win_rel_rows(int mb) {
  return (mb + 2 + kWinChunk - 1) / kWinChunk * kWinChunk;
}

// Shared memory of the window kernel: the Stage-1 tile; Stage 2 and 3 reuse it.
template <class Tin, class Tred, class T>
struct WinSmem {
  static constexpr size_t kTile = Tile<Tin, kWinChunk>::kBytesPerWarp;
  static constexpr size_t kRelBuf = (size_t)3 * kWinChunk * 32 * sizeof(Tred);  // one chunk
  static constexpr size_t kXTile = (size_t)32 * Tile<Tin, kWinChunk>::kStride * sizeof(Tin);
  static constexpr size_t kStage3 = 2 * kRelBuf + kXTile;
  static constexpr size_t kRed = (size_t)4 * 64 * sizeof(T);
  static constexpr size_t kBytes = kTile > kStage3 ? (kTile > kRed ? kTile : kRed)
                                                   : (kStage3 > kRed ? kStage3 : kRed);
};

// One warp per window (grid: the windows).  n > kBaseMax; R kept rows and h
// halo rows with R + 2 h = 32 mb; rel: win_rel_rows(mb) * 96 elements of
// Tred per window; bound_max zeroed before the launch; dmax: the system's
// range codes (double-float) or null.  kVec16: arrays 16-byte aligned, and
// mb, R, h multiples of the 16-byte vector.
template <class Ar, class Tin, class Tred, bool kVec16>
__global__ void __launch_bounds__(32)
    k_wsolve(int64_t n, int R, int h, int mb, const Tin* __restrict__ a,
             const Tin* __restrict__ b, const Tin* __restrict__ c, const Tin* __restrict__ d,
             Tin* __restrict__ x, Tred* __restrict__ rel, float tol,
             unsigned* __restrict__ bound_max, int* __restrict__ status,
             unsigned* __restrict__ dmax) {
  using T = typename Ar::T;
  constexpr int C = kWinChunk;
  using TL = Tile<Tin, C>;
  using SM = WinSmem<Tin, Tred, T>;
  constexpr int V = TL::kVec;
  constexpr unsigned kAll = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tin* tile = reinterpret_cast<Tin*>(smem_raw);
  const int lane = threadIdx.x;
  const int64_t w = blockIdx.x;
  WinGeom G;
  G.init(n, R, h, w);
  int64_t b0, b1;
  G.block(mb, h, lane, b0, b1);
  const int L = (int)(b1 - b0);
  const bool active = L > 0;
  const bool cut_first = active && b0 == G.e0;  // the window's first row: its a is cut
  const bool cut_last = active && b1 == G.e1;   // the window's last row: its c is cut
  const int nch = __reduce_max_sync(kAll, (unsigned)((L + C - 1) / C));
  // every lane a full block of mb rows, mb a whole number of chunks: the
  // chunks run through one unrolled body
  const bool uniform = __all_sync(kAll, L == mb) && mb % C == 0;
  Tred* const wrel = rel + (size_t)w * win_rel_rows(mb) * 96;

  const Tin* const srcs[4] = {a, b, c, d};
  WinPieces<Tin, C> pm;
  pm.init(G, mb, h, lane);
  load_chunk<Tin, C, kVec16>(tile, srcs, 4, pm, 0);
  cp_async_commit();

  // ---- Stage 1: divided form.  Virtual state before row 1 (relation
  // x_0 = f): c' = 0, g' = 0, alpha' = -1; first interior unknown
  // x_1 = P - Q f - S x_{j+1} with P = Q = 0, S = -1.
  T cp = Ar::zero(), gp = Ar::zero(), ap = Ar::neg(Ar::one());
  T P = Ar::zero(), Q = Ar::zero(), S = Ar::neg(Ar::one());
  T a0 = Ar::zero(), b0v = Ar::one(), c0 = Ar::zero(), d0 = Ar::zero();
  T beta = Ar::one(), g = Ar::zero(), al = Ar::zero(), clast = Ar::zero();
  bool bad = false;
  RowChk chk;
  float qmax = 0.0f;
  unsigned bminw = 0x7FFFFFFFu;  // smallest |b| (high word of the fp64 / fp32 bits)

  // dominance of one row (cut couplings 0): (|a| + |c|) / |b| from the
  // arithmetic's values, the reciprocal approximate (the bound widens q)
  auto dominance = [&](const T& av, const T& bv, const T& cv) {
    if constexpr (std::is_same<T, double>::value) {
      // native fp64 rows are not scaled: their ratio from the scaled split
      qmax = fmaxf(qmax, win_row_q(av, bv, cv));
    } else {
      float r;
      asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(fabsf(lead_f32(bv))));
      qmax = fmaxf(qmax, (fabsf(lead_f32(av)) + fabsf(lead_f32(cv))) * r);
    }
  };
  auto bmin_raw = [&](Tin bin) {
    unsigned wv;
    if constexpr (sizeof(Tin) == 8) wv = (unsigned)__double2hiint((double)bin) & 0x7FFFFFFFu;
    else wv = __float_as_uint((float)bin) & 0x7FFFFFFFu;
    bminw = min(bminw, wv);
  };
  auto interior = [&](int j, const T& av, const T& bv, const T& cv, const T& dv) {
    beta = Ar::sub_mul_dom(bv, av, cp);
    bad |= Ar::bad_pivot(beta);
    const T r = Ar::rcp(beta);
    gp = Ar::mul(Ar::sub_mul(dv, av, gp), r);
    ap = Ar::mul(Ar::mul_neg_nn(av, ap), r);
    cp = Ar::mul(cv, r);
    P = Ar::sub_mul_nn(P, S, gp);
    Q = Ar::sub_mul_nn(Q, S, ap);
    S = Ar::mul_neg_nn(S, cp);
    Tred* o = wrel + (size_t)j * 96 + lane;
    Ar::to(o[0], cp);
    Ar::to(o[32], gp);
    Ar::to(o[64], ap);
  };
  auto last_row = [&](const T& av, const T& bv, const T& cv, const T& dv) {
    beta = Ar::sub_mul_dom(bv, av, cp);
    g = Ar::sub_mul(dv, av, gp);
    al = Ar::mul_neg_nn(av, ap);
    clast = cv;
  };
  auto renorm = [&]() {
    P = Ar::norm(P);
    Q = Ar::norm(Q);
    S = Ar::norm(S);
  };

  for (int ch = 0; ch < nch; ++ch) {
    const int row0 = ch * C;
    if (ch + 1 < nch)
      load_chunk<Tin, C, kVec16>(tile + ((ch + 1) & 1) * TL::kBuf, srcs, 4, pm, row0 + C);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    const Tin* t = tile + (ch & 1) * TL::kBuf + lane * TL::kStride;
    if (uniform) {
      const bool first = ch == 0, last = ch == nch - 1;
#pragma unroll
      for (int r = 0; r < C; r += V) {
        const Vec16<Tin> xa = lds16(t + r), xb = lds16(t + TL::kArr + r),
                         xc = lds16(t + 2 * TL::kArr + r), xd = lds16(t + 3 * TL::kArr + r);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int rr = r + v;
          const bool is_f = rr == 0 && first, is_l = rr == C - 1 && last;
          const Tin ain = (is_f && cut_first) ? Tin{} : xa.v[v];
          const Tin cin = (is_l && cut_last) ? Tin{} : xc.v[v];
          T av, bv, cv, dv;
          Ar::template row<true>(ain, xb.v[v], cin, xd.v[v], av, bv, cv, dv, chk);
          dominance(av, bv, cv);
          bmin_raw(xb.v[v]);
          if (is_f) {
            a0 = av; b0v = bv; c0 = cv; d0 = dv;
          } else if (is_l) {
            last_row(av, bv, cv, dv);
          } else {
            interior(row0 + rr, av, bv, cv, dv);
          }
        }
      }
    } else {
#pragma unroll 1
      for (int r = 0; r < C; ++r) {
        const int row = row0 + r;
        if (row < L) {
          const bool is_f = row == 0, is_l = row == L - 1;
          const Tin ain = (is_f && cut_first) ? Tin{} : t[r];
          const Tin cin = (is_l && cut_last) ? Tin{} : t[2 * TL::kArr + r];
          T av, bv, cv, dv;
          Ar::template row<true>(ain, t[TL::kArr + r], cin, t[3 * TL::kArr + r], av, bv, cv, dv,
                                 chk);
          dominance(av, bv, cv);
          bmin_raw(t[TL::kArr + r]);
          if (is_f) {
            a0 = av; b0v = bv; c0 = cv; d0 = dv;
          } else if (is_l) {
            last_row(av, bv, cv, dv);
          } else {
            interior(row, av, bv, cv, dv);
          }
        }
      }
    }
    renorm();
    __syncwarp();  // the buffer is refilled by the next iteration's copies
  }
  bad |= active && Ar::bad_pivot(beta);
  if (active && chk.range_bad()) atomicOr(status, ST_RANGE);
  bad |= active && chk.b_bad();
  if (dmax) codes_raise_warp(dmax, 0, active, chk);

  // ---- Stage 2: the window's 64 reduced rows, lane l's rows 2l (first:
  // l_{l-1}, f_l, l_l) and 2l + 1 (last: f_l, l_l, f_{l+1}); an empty block
  // gives two identity rows.  Parallel cyclic reduction in the warp.
  cp_async_wait<0>();
  __syncwarp();
  T* sa = reinterpret_cast<T*>(smem_raw);
  T* sb = sa + 64;
  T* sc = sb + 64;
  T* sd = sc + 64;
  if (active) {
    sa[2 * lane] = cut_first ? Ar::zero() : a0;
    sb[2 * lane] = Ar::sub_mul(b0v, c0, Q);
    sc[2 * lane] = Ar::neg(Ar::mul(c0, S));
    sd[2 * lane] = Ar::sub_mul(d0, c0, P);
    sa[2 * lane + 1] = al;
    sb[2 * lane + 1] = beta;
    sc[2 * lane + 1] = cut_last ? Ar::zero() : clast;
    sd[2 * lane + 1] = g;
  } else {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      sa[2 * lane + k] = Ar::zero(); sb[2 * lane + k] = Ar::one();
      sc[2 * lane + k] = Ar::zero(); sd[2 * lane + k] = Ar::zero();
    }
  }
  __syncwarp();
  for (int s = 1; s < 64; s <<= 1) {
    T na[2], nbv[2], nc[2], nd[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int i = 2 * lane + k;
      const int im = i - s, ip = i + s;
      const T am = im >= 0 ? sa[im] : Ar::zero(), bm = im >= 0 ? sb[im] : Ar::one();
      const T cm = im >= 0 ? sc[im] : Ar::zero(), dm = im >= 0 ? sd[im] : Ar::zero();
      const T ap2 = ip < 64 ? sa[ip] : Ar::zero(), bp = ip < 64 ? sb[ip] : Ar::one();
      const T cp2 = ip < 64 ? sc[ip] : Ar::zero(), dp = ip < 64 ? sd[ip] : Ar::zero();
      bad |= Ar::bad_pivot(bm) | Ar::bad_pivot(bp);
      const T k1 = Ar::mul(sa[i], Ar::rcp(bm));
      const T k2 = Ar::mul(sc[i], Ar::rcp(bp));
      na[k] = Ar::neg(Ar::mul(am, k1));
      nc[k] = Ar::neg(Ar::mul(cp2, k2));
      nbv[k] = Ar::sub_mul(Ar::sub_mul(sb[i], cm, k1), ap2, k2);
      nd[k] = Ar::sub_mul(Ar::sub_mul(sd[i], dm, k1), dp, k2);
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int i = 2 * lane + k;
      sa[i] = na[k]; sb[i] = nbv[k]; sc[i] = nc[k]; sd[i] = nd[k];
    }
    __syncwarp();
  }
  bad |= Ar::bad_pivot(sb[2 * lane]) | Ar::bad_pivot(sb[2 * lane + 1]);
  const T f = Ar::mul(sd[2 * lane], Ar::rcp(sb[2 * lane]));
  const T l = Ar::mul(sd[2 * lane + 1], Ar::rcp(sb[2 * lane + 1]));
  __syncwarp();  // the reduced rows are read; Stage 3 reuses the memory

  // ---- Stage 3: bottom-up through the relations, chunk by chunk; each
  // chunk's relations (3 x 8 rows x 32 lanes, contiguous) staged by cp.async
  Tred* rbuf = reinterpret_cast<Tred*>(smem_raw);                      // [2][3 * C * 32]
  Tin* xt = reinterpret_cast<Tin*>(smem_raw + 2 * SM::kRelBuf);        // [32][kStride]
  Tin* xs = xt + lane * TL::kStride;
  constexpr int kRelPieces = (int)(SM::kRelBuf / 16);
  auto load_rel = [&](Tred* dst, int ch) {
    const unsigned char* src = reinterpret_cast<const unsigned char*>(wrel + (size_t)ch * C * 96);
    unsigned char* dd = reinterpret_cast<unsigned char*>(dst);
    for (int i = lane; i < kRelPieces; i += 32) cp_async<16>(dd + 16 * i, src + 16 * i);
  };
  load_rel(rbuf, nch - 1);
  cp_async_commit();
  T xnext = l;
  bool oob = false;
  for (int it = 0; it < nch; ++it) {
    const int ch = nch - 1 - it;
    const int row0 = ch * C;
    if (ch > 0) load_rel(rbuf + ((it + 1) & 1) * (3 * C * 32), ch - 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    const Tred* rb = rbuf + (it & 1) * (3 * C * 32) + lane;
    if (uniform) {
      // every lane the same rows: only the block's first row (chunk 0) and
      // last row (last chunk) take the interface values; one unrolled body,
      // x out through 16-byte shared stores
      const bool first = ch == 0, last = ch == nch - 1;
      Tin xo[C];
#pragma unroll
      for (int r = C - 1; r >= 0; --r) {
        T xr;
        if (r == C - 1 && last) {
          xr = l;
        } else if (r == 0 && first) {
          xr = f;
        } else {
          const T cr = Ar::from(rb[(r * 3 + 0) * 32]);
          const T gr = Ar::from(rb[(r * 3 + 1) * 32]);
          const T ar = Ar::from(rb[(r * 3 + 2) * 32]);
          xr = Ar::sub_mul(Ar::sub_mul_nn(gr, ar, f), cr, xnext);
          xnext = xr;
        }
        Ar::to(xo[r], xr);
        oob |= Ar::out_bad(xo[r]);
      }
#pragma unroll
      for (int r = 0; r < C; r += V) {
        Vec16<Tin> wv;
#pragma unroll
        for (int v = 0; v < V; ++v) wv.v[v] = xo[r + v];
        *reinterpret_cast<float4*>(xs + r) = *reinterpret_cast<const float4*>(&wv);
      }
    } else {
#pragma unroll 1
      for (int r = C - 1; r >= 0; --r) {
        const int row = row0 + r;
        if (row < L) {
          T xr;
          if (row == L - 1) {
            xr = l;
          } else if (row == 0) {
            xr = f;
          } else {
            const T cr = Ar::from(rb[(r * 3 + 0) * 32]);
            const T gr = Ar::from(rb[(r * 3 + 1) * 32]);
            const T ar = Ar::from(rb[(r * 3 + 2) * 32]);
            xr = Ar::sub_mul(Ar::sub_mul_nn(gr, ar, f), cr, xnext);
            xnext = xr;
          }
          Tin xo;
          Ar::to(xo, xr);
          oob |= Ar::out_bad(xo);
          xs[r] = xo;
        }
      }
    }
    __syncwarp();
    store_kept<Tin, C, kVec16>(x, xt, pm, row0, G.k0, G.k1);
    __syncwarp();  // the buffers are refilled by the next iteration's copies
  }
  // the relation slice is dead: drop it from L2 without a write-back
  {
    const size_t bytes = (size_t)win_rel_rows(mb) * 96 * sizeof(Tred);
    const unsigned char* base = reinterpret_cast<const unsigned char*>(wrel);
    for (size_t o = (size_t)lane * 128; o < bytes; o += 32 * 128) discard_l2(base + o);
  }
  if (active && bad) atomicOr(status, ST_BAD_PIVOT);
  if (active && oob) atomicOr(status, ST_RANGE);

  // ---- the window's truncation bound
  const unsigned qbits = __reduce_max_sync(kAll, __float_as_uint(qmax));
  const unsigned bw = __reduce_min_sync(kAll, active ? bminw : 0x7FFFFFFFu);
  if (lane == 0) {
    const float q = __fmul_ru(__uint_as_float(qbits), 1.0f + 9.5367431640625e-07f);
    // |a_cut| / min |b| and |c_cut| / min |b|, rounded up (scale-free, so a
    // system scaled anywhere in the input's range gets the same bound);
    // min |b| from the high words, rounded down
    float ra = 0.0f, rc = 0.0f;
    if constexpr (sizeof(Tin) == 8) {
      const double bmd = __hiloint2double((int)bw, 0);
      if (G.e0 > 0) ra = __double2float_ru(__ddiv_ru(fabs((double)a[G.e0]), bmd));
      if (G.e1 < n) rc = __double2float_ru(__ddiv_ru(fabs((double)c[G.e1 - 1]), bmd));
    } else {
      const float bmf = __uint_as_float(bw);
      if (G.e0 > 0) ra = __fdiv_ru(fabsf((float)a[G.e0]), bmf);
      if (G.e1 < n) rc = __fdiv_ru(fabsf((float)c[G.e1 - 1]), bmf);
    }
    float eps;
    if (ra == 0.0f && rc == 0.0f) {
      eps = 0.0f;  // nothing cut
    } else if (!(q < 1.0f) || !(ra < __int_as_float(0x7f800000)) ||
               !(rc < __int_as_float(0x7f800000))) {
      eps = __int_as_float(0x7f800000);
    } else {
      const float num = __fadd_ru(__fmul_ru(ra, powf(q, (float)(G.k0 - G.e0))),
                                  __fmul_ru(rc, powf(q, (float)(G.e1 - G.k1))));
      eps = __fdiv_ru(num, __fsub_rd(1.0f, q)) * (1.0f + 1e-5f);
    }
    atomicMax(bound_max, __float_as_uint(eps));
    if (!(eps <= tol)) atomicOr(status, ST_NO_CONVERGENCE);
  }
}

}  // namespace tps
