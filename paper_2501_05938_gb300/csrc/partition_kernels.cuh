// Stage 1, Stage 3 and the small-system solve of the tridiagonal partition
// method (Sec. 1 and Sec. 2.2 of the paper: per-block elimination onto the
// interface unknowns, a reduced interface solve, per-block recovery).
//
// System: a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i]; a[0], c[n-1] unused.
// Blocks: block k owns rows k*m .. k*m + L_k - 1, L_k = m except the last
// block, whose length Llast lies in [2, m + 1] (a one-row tail is merged into
// the block before it).  The first and last row of each block are its
// interface unknowns f_k and l_k; the reduced system in (f_0, l_0, f_1, ...)
// is tridiagonal: row 2k is block k's "first" equation in (l_{k-1}, f_k, l_k)
// and row 2k+1 its "last" equation in (f_k, l_k, f_{k+1}).
//
// GPU mapping.  One lane owns one block and sweeps it serially (the
// recurrences are first-order); a warp owns 32 consecutive blocks and a CTA
// W warps.  The warp streams its blocks through shared memory in chunks of R
// rows, double buffered: for each of a, b, c, d the warp copies the chunk's
// rows of its 32 blocks with cp.async in 16-byte pieces, consecutive lanes
// taking consecutive pieces of one block (64 contiguous bytes per block for
// fp64), so each copy instruction moves 512 coalesced bytes.  Per-lane piece
// offsets are computed once per kernel.  In shared memory each block's rows
// sit in a slot padded to R + 16/sizeof(element) elements, so the 128-bit
// loads with which a lane reads its own block hit distinct banks across a
// quarter-warp.  Where pointers are not 16-byte aligned (or m is not a
// multiple of the 16-byte vector) the same copies go element by element.
//
// Stage 1 is a single top-down sweep per block.  Writing the interior
// relation after row j as  beta_j x_j + c_j x_{j+1} = g_j - alpha_j f  (a
// forward elimination that keeps f symbolic), the last reduced equation is
// the relation after the block's last row, (alpha, beta, c, g) on
// (f_k, l_k, f_{k+1}).  The first reduced equation needs the first interior
// unknown as a function of f_k and l_k; instead of a second, bottom-up
// sweep, the sweep carries x_1 = P - Q f - S x_{j+1} along, which costs four
// multiply-adds per row and no extra reciprocal.  At every chunk boundary
// the normalised relation x_j = (g_j - alpha_j f - c_j x_{j+1}) / beta_j is
// written out as a checkpoint (c/beta, g/beta, alpha/beta).
//
// Stage 3 walks each block's chunks bottom-up.  A chunk restarts the forward
// elimination from its checkpoint (with f now known), keeps the R pivots and
// right-hand sides in registers, and back-substitutes from the x of the row
// below it (l_k for the last chunk).  The chunk's x goes back through the
// shared-memory slots and out with the same coalesced piece mapping.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "arith.cuh"

namespace tps {

// ------------------------------------------------------------------ geometry
struct Level {
  int64_t n;        // rows
  int64_t p;        // blocks
  int64_t k_begin;  // blocks this launch processes: [k_begin, k_end)
  int64_t k_end;
  const int64_t* bnd;  // batched systems: first rows of systems 1.., sorted (device)
  int64_t nbnd;        // number of such rows (0: one system)
  int32_t m;        // nominal block length
  int32_t llast;    // length of block p-1, in [2, m+1]
  int32_t ncap;     // checkpoint slots per block
  int32_t pad;
  // level 0 of fp64 inputs in narrower arithmetic: per system (nbnd + 1
  // of them) the kCodes range codes of its rows (RowChk), raised by Stage 1
  // with atomicMax; null elsewhere
  unsigned* dmax;
};

__device__ __forceinline__ int block_len(const Level& lv, int64_t k) {
  return k == lv.p - 1 ? lv.llast : lv.m;
}

// Systems packed back to back are solved as one system whose couplings are
// cut at every system boundary: a of a system's first row and c of its last
// row are taken as 0 (they are never read).  A block may straddle
// boundaries; its recurrences then decouple exactly there.  Each lane keeps
// the boundaries that touch its block, bnd[first .. first+cnt).
struct Bounds {
  const int64_t* bnd;
  int64_t first;
  int cnt;
  // first index i with bnd[i] >= v
  __device__ __forceinline__ static int64_t lower(const int64_t* b, int64_t nb, int64_t v) {
    int64_t lo = 0, hi = nb;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (b[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
  }
  // boundaries o with start <= o <= start + len (a start row, or the row
  // after the block's last row)
  __device__ __forceinline__ void init(const Level& lv, int64_t start, int len, bool active) {
    bnd = lv.bnd;
    first = 0;
    cnt = 0;
    if (lv.nbnd == 0 || !active) return;
    first = lower(lv.bnd, lv.nbnd, start);
    cnt = (int)(lower(lv.bnd, lv.nbnd, start + len + 1) - first);
  }
  // a boundary within rows [g0, g0 + rows] (the chunk, or its successor row)
  __device__ __forceinline__ bool touches(int64_t g0, int rows) const {
    for (int j = 0; j < cnt; ++j) {
      const int64_t o = bnd[first + j];
      if (o >= g0 && o <= g0 + rows) return true;
    }
    return false;
  }
  __device__ __forceinline__ bool is(int64_t row) const {
    for (int j = 0; j < cnt; ++j)
      if (bnd[first + j] == row) return true;
    return false;
  }
};

// Status bits written into the device status word.
enum : int { ST_BAD_PIVOT = 1, ST_NO_CONVERGENCE = 2, ST_TIMEOUT = 4, ST_RANGE = 8 };

// Range codes of packed systems: three words per system (RowChk's dcode,
// ecode, fcode maxima).  Raise system `sys`'s codes to v (an atomic only
// where that would change a code; the entries are read from L2).
constexpr int kCodes = 3;
__device__ __forceinline__ void code_raise(unsigned* p, unsigned v) {
  if (v != 0u && __ldcg(p) < v) atomicMax(p, v);
}
__device__ __forceinline__ void codes_raise(unsigned* dmax, int64_t sys, unsigned dc,
                                            unsigned ec, unsigned fc) {
  unsigned* p = dmax + kCodes * sys;
  code_raise(p, dc);
  code_raise(p + 1, ec);
  code_raise(p + 2, fc);
}
// The warp's codes: one set of atomics per warp where every lane is in the
// same system (always for a single system), else per lane.
__device__ __forceinline__ void codes_raise_warp(unsigned* dmax, int64_t sys, bool active,
                                                 const RowChk& k) {
  const unsigned dc = active ? k.dcode() : 0u, ec = active ? k.ecode : 0u,
                 fc = active ? k.fcode() : 0u;
  const int64_t sys0 = __shfl_sync(0xffffffffu, sys, 0);
  if (__all_sync(0xffffffffu, !active || sys == sys0)) {
    const unsigned wd = __reduce_max_sync(0xffffffffu, dc);
    const unsigned we = __reduce_max_sync(0xffffffffu, ec);
    const unsigned wf = __reduce_max_sync(0xffffffffu, fc);
    if ((threadIdx.x & 31) == 0) codes_raise(dmax, sys0, wd, we, wf);
  } else if (active) {
    codes_raise(dmax, sys, dc, ec, fc);
  }
}

// After every row of the level-0 system has been loaded: flag ST_RANGE for
// each system whose codes are out of range (range_codes_bad), and clear the
// codes for the next solve.  One CTA.
static __global__ void __launch_bounds__(256)
    k_dcode_check(unsigned* __restrict__ dmax, int64_t count, int* __restrict__ status) {
  bool bad = false;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
    unsigned* p = dmax + kCodes * i;
    bad |= range_codes_bad(p[0], p[1], p[2]);
    p[0] = p[1] = p[2] = 0u;
  }
  if (bad) atomicOr(status, ST_RANGE);
}

// ------------------------------------------------------------------ cp.async
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
  const uint32_t s = smem_u32(smem_dst);
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
  } else if constexpr (BYTES == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
  } else {
    static_assert(BYTES == 4, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------------------ warp tile
// NA arrays per buffer: a, b, c, d, and for a refinement step (RefineIO) the
// current x as a fifth.
template <class Tin, int R, int NA = 4>
struct Tile {
  static constexpr int kVec = 16 / (int)sizeof(Tin);  // elements per 16-byte piece
  static_assert(R % kVec == 0, "chunk rows must fill 16-byte pieces");
  static constexpr int kPieces = R / kVec;            // pieces per block and chunk
  static constexpr int kStride = R + kVec;            // padded block slot (16-byte multiple)
  static constexpr int kArr = 32 * kStride;           // one array of one buffer
  static constexpr int kBuf = NA * kArr;
  static constexpr size_t kBytesPerWarp = sizeof(Tin) * 2 * kBuf;
};

// Stage 3 also prefetches each chunk's checkpoint (three values per block)
// with the chunk: per buffer, 3 x 32 values after the warp's two buffers.
template <class Tin, class Tred, int R, int NA = 4>
struct Tile3 : Tile<Tin, R, NA> {
  static constexpr size_t kCkBytesPerBuf = 3 * 32 * sizeof(Tred);
  static constexpr size_t kBytesPerWarp = Tile<Tin, R, NA>::kBytesPerWarp + 2 * kCkBytesPerBuf;
};

// One correction step of mixed-precision iterative refinement, fused into
// the level-0 sweeps (kRef kernels; fp64 arrays).  Stage 1 forms the
// residual r = d - A x of the current iterate in fp64 while it streams the
// rows, eliminates with r as the right-hand side and writes r out; Stage 3,
// given r as its right-hand side, adds the correction delta to x in place
// and raises max2[0] = max |delta|, max2[1] = max |x + delta|, each as the
// bit pattern of a non-negative double (which orders like the value; a NaN
// ranks above +inf).
struct RefineIO {
  const double* x;          // Stage 1: the current iterate (read with its neighbours)
  double* r;                // Stage 1: the residual, written
  unsigned long long* max2; // Stage 3: the two maxima (zeroed before the launch)
};

// Pieces of the current x a Stage-1 refinement chunk needs: its R rows and
// the next piece (the row below the chunk), i.e. kPieces + 1 pieces filling
// the block's padded slot; piece q = lane + 32 j (j <= kPieces) is piece
// q % (kPieces + 1) of block q / (kPieces + 1).
template <class Tin, int R>
struct XPieceMap {
  using TL = Tile<Tin, R>;
  static constexpr int kP = TL::kPieces + 1;
  int64_t goff[kP];
  int soff[kP];
  int row[kP];
  int len[kP];
  __device__ __forceinline__ void init(const Level& lv, int64_t k0, int nb, int lane) {
#pragma unroll
    for (int j = 0; j < kP; ++j) {
      const int q = lane + 32 * j;
      const int blk = q / kP;
      const int pc = q % kP;
      row[j] = pc * TL::kVec;
      len[j] = blk < nb ? block_len(lv, k0 + blk) : 0;
      goff[j] = (k0 + blk) * (int64_t)lv.m + row[j];
      soff[j] = blk * TL::kStride + row[j];
    }
  }
};

// 16 bytes of consecutive rows (one 128-bit shared access).
template <class Tin>
struct Vec16 {
  Tin v[16 / sizeof(Tin)];
};
template <class Tin>
__device__ __forceinline__ Vec16<Tin> lds16(const Tin* p) {
  Vec16<Tin> r;
  *reinterpret_cast<float4*>(&r) = *reinterpret_cast<const float4*>(p);
  return r;
}

// The pieces lane `lane` copies for every array: piece q = lane + 32 j
// (j < kPieces) is piece q % kPieces of block q / kPieces of the warp.
template <class Tin, int R>
struct PieceMap {
  using TL = Tile<Tin, R>;
  int64_t goff[TL::kPieces];  // element offset of the piece in the arrays (chunk 0)
  int soff[TL::kPieces];      // element offset in a buffer's array
  int row[TL::kPieces];       // first row of the piece within its block (chunk 0)
  int len[TL::kPieces];       // length of the piece's block, 0 past the last block
  __device__ __forceinline__ void init(const Level& lv, int64_t k0, int nb, int lane);
};

template <class Tin, int R>
__device__ __forceinline__ void PieceMap<Tin, R>::init(const Level& lv, int64_t k0, int nb,
                                                       int lane) {
#pragma unroll
  for (int j = 0; j < TL::kPieces; ++j) {
    const int q = lane + 32 * j;
    const int blk = q / TL::kPieces;
    const int pc = q % TL::kPieces;
    row[j] = pc * TL::kVec;
    len[j] = blk < nb ? block_len(lv, k0 + blk) : 0;
    goff[j] = (k0 + blk) * (int64_t)lv.m + row[j];
    soff[j] = blk * TL::kStride + row[j];
  }
}

// Copy rows [row0, row0 + R) of the warp's blocks (clipped to each block's
// length) of src[0..n_arr) into the buffer's arrays.  kVec16: whole pieces
// go as one 16-byte copy (arrays 16-byte aligned, m a multiple of kVec);
// otherwise, and for a block's ragged last piece, element by element.
template <class Tin, int R, bool kVec16, class PM>
__device__ __forceinline__ void load_chunk(Tin* buf, const Tin* const* src, int n_arr,
                                           const PM& pm, int row0) {
  using TL = Tile<Tin, R>;
#pragma unroll
  for (int j = 0; j < TL::kPieces; ++j) {
    const int avail = pm.len[j] - (row0 + pm.row[j]);  // rows of this piece in its block
    const int64_t g = pm.goff[j] + row0;
    if (kVec16 && avail >= TL::kVec) {
      for (int t = 0; t < n_arr; ++t) cp_async<16>(buf + t * TL::kArr + pm.soff[j], src[t] + g);
    } else if (avail > 0) {
#pragma unroll
      for (int v = 0; v < TL::kVec; ++v)
        if (v < avail)
          for (int t = 0; t < n_arr; ++t)
            cp_async<sizeof(Tin)>(buf + t * TL::kArr + pm.soff[j] + v, src[t] + g + v);
    }
  }
}

// Write rows [row0, row0 + R) of the warp's blocks from the buffer's first
// array to x (same piece mapping as the loads).
template <class Tin, int R, bool kVec16>
__device__ __forceinline__ void store_chunk(Tin* __restrict__ x, const Tin* buf,
                                            const PieceMap<Tin, R>& pm, int row0) {
  using TL = Tile<Tin, R>;
#pragma unroll
  for (int j = 0; j < TL::kPieces; ++j) {
    const int avail = pm.len[j] - (row0 + pm.row[j]);
    const int64_t g = pm.goff[j] + row0;
    if (kVec16 && avail >= TL::kVec) {
      *reinterpret_cast<float4*>(x + g) = *reinterpret_cast<const float4*>(buf + pm.soff[j]);
    } else if (avail > 0) {
#pragma unroll
      for (int v = 0; v < TL::kVec; ++v)
        if (v < avail) x[g + v] = buf[pm.soff[j] + v];
    }
  }
}

// Rows [row0, row0 + R] of the current x for the warp's blocks: every row up
// to and including the one below the block (the next block's first row),
// clipped to the array's n rows.
template <class Tin, int R, bool kVec16>
__device__ __forceinline__ void load_xchunk(Tin* buf, const Tin* x, const XPieceMap<Tin, R>& xm,
                                            int row0, int64_t n) {
  using TL = Tile<Tin, R>;
#pragma unroll
  for (int j = 0; j < XPieceMap<Tin, R>::kP; ++j) {
    if (xm.len[j] == 0) continue;
    const int64_t g = xm.goff[j] + row0;
    const int64_t avail = min((int64_t)(xm.len[j] + 1 - (row0 + xm.row[j])), n - g);
    if (kVec16 && avail >= TL::kVec) {
      cp_async<16>(buf + xm.soff[j], x + g);
    } else if (avail > 0) {
#pragma unroll
      for (int v = 0; v < TL::kVec; ++v)
        if (v < avail) cp_async<sizeof(Tin)>(buf + xm.soff[j] + v, x + g + v);
    }
  }
}

// r = d - (a x_{i-1} + b x_i + c x_{i+1}) in fp64 (a and c already cut to
// zero where a coupling does not exist, and the matching x passed as 0).
__device__ __forceinline__ double residual_row(double a, double b, double c, double d, double xm,
                                               double x0, double xp) {
  double r = fma(-b, x0, d);
  r = fma(-a, xm, r);
  return fma(-c, xp, r);
}
// |v|'s bit pattern from integer operations on the two halves (masking the
// sign of the 64-bit pattern is compiled as an fp64 absolute value, an
// instruction of the slow fp64 pipe: measured 2 of the 3 fp64 instructions
// per row of the refinement's Stage 3)
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  const unsigned hi = (unsigned)__double2hiint(v) & 0x7FFFFFFFu;
  const unsigned lo = (unsigned)__double2loint(v);
  return ((unsigned long long)hi << 32) | lo;
}

// chunks the warp iterates: the longest block of the warp decides
__device__ __forceinline__ int warp_chunks(const Level& lv, int64_t k0, int nb, int R) {
  const int lmax = (k0 + nb == lv.p) ? max(lv.m, lv.llast) : lv.m;
  return (lmax + R - 1) / R;
}
// shortest block among the warp's active lanes
__device__ __forceinline__ int warp_lmin(const Level& lv, int64_t k0, int nb) {
  return (k0 + nb == lv.p) ? min(lv.m, lv.llast) : lv.m;
}
// the block length every active lane of the warp has, or 0 if they differ
__device__ __forceinline__ int warp_luni(const Level& lv, int64_t k0, int nb) {
  return (k0 + nb == lv.p) ? (lv.llast == lv.m ? lv.m : 0) : lv.m;
}

// Chunks that every active lane sees the same way run unrolled: all rows
// interior (kMid), the block's first row f and then interior rows (kFirst,
// chunk 0), or interior rows and then the block's last row l (kLast, when
// every lane's block ends with the chunk).  Any other chunk (a ragged last
// block, a packed-system boundary in or next to the chunk) goes row by row.
enum ChunkKind : int { kSlow = -1, kMid = 0, kFirst = 1, kLast = 2 };
__device__ __forceinline__ int chunk_kind(int ch, int row0, int R, int lmin, int luni,
                                          bool clean) {
  if (!clean) return kSlow;
  if (ch >= 1 && row0 + R <= lmin - 1) return kMid;
  if (ch == 0 && R <= lmin - 1) return kFirst;
  if (ch >= 1 && luni > 0 && row0 + R == luni) return kLast;
  return kSlow;
}

// ------------------------------------------------------------------ Stage 1
// Chunk buffers per warp in Stage 1's copy pipeline (2: the next chunk is
// copied while one is processed).
#ifndef TPS_STAGE1_STAGES
#define TPS_STAGE1_STAGES 2
#endif
constexpr int kS1Stages = TPS_STAGE1_STAGES;
static_assert(kS1Stages >= 2 && kS1Stages <= 4, "Stage-1 pipeline depth");
// Shared memory of one Stage-1 warp (NA arrays per buffer).
template <class Tin, int R, int NA = 4>
constexpr size_t stage1_smem_per_warp() {
  return Tile<Tin, R, NA>::kBytesPerWarp / 2 * kS1Stages;
}

// R rows per chunk; a checkpoint every K rows (K the chunk length of
// Stage 3; one of R and K divides the other).  kRef: a refinement step
// (RefineIO), the right-hand side being the residual of rf.x.
template <class Ar, class Tin, class Tred, int R, int K, int W, bool kVec16, bool kRef = false>
__global__ void __launch_bounds__(W * 32)
    k_stage1(Level lv, const Tin* __restrict__ a, const Tin* __restrict__ b,
             const Tin* __restrict__ c, const Tin* __restrict__ d, Tred* __restrict__ ra,
             Tred* __restrict__ rb, Tred* __restrict__ rc, Tred* __restrict__ rd,
             Tred* __restrict__ ck_gam, Tred* __restrict__ ck_y, Tred* __restrict__ ck_v,
             int* __restrict__ status, RefineIO rf = {}) {
  using T = typename Ar::T;
  using TL = Tile<Tin, R, kRef ? 5 : 4>;
  constexpr int V = TL::kVec;
  static_assert(!kRef || std::is_same<Tin, double>::value, "refinement steps are fp64");
  static_assert(R % K == 0 || K % R == 0, "chunk rows and checkpoint spacing must nest");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k0 = lv.k_begin + ((int64_t)blockIdx.x * W + warp) * 32;
  if (k0 >= lv.k_end) return;
  const int nb = (int)(lv.k_end - k0 < 32 ? lv.k_end - k0 : 32);
  const int64_t k = k0 + lane;
  const bool active = lane < nb;
  const int L = active ? block_len(lv, k) : 0;
  const int nch = warp_chunks(lv, k0, nb, R);
  const int lmin = warp_lmin(lv, k0, nb);
  const int luni = warp_luni(lv, k0, nb);

  Tin* tile = reinterpret_cast<Tin*>(smem_raw) + warp * kS1Stages * TL::kBuf;
  const Tin* const srcs[4] = {a, b, c, d};
  PieceMap<Tin, R> pm;
  pm.init(lv, k0, nb, lane);
  XPieceMap<Tin, R> xpm;
  if constexpr (kRef) xpm.init(lv, k0, nb, lane);
  // chunk c goes to buffer c % kS1Stages, one commit group per chunk
  auto fetch = [&](int c) {
    if (c < nch) {
      Tin* buf = tile + (c % kS1Stages) * TL::kBuf;
      load_chunk<Tin, R, kVec16>(buf, srcs, 4, pm, c * R);
      if constexpr (kRef)
        load_xchunk<Tin, R, kVec16>(buf + 4 * TL::kArr, (const Tin*)rf.x, xpm, c * R, lv.n);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int c = 0; c < kS1Stages - 1; ++c) fetch(c);
  const int64_t start = k * (int64_t)lv.m;
  Bounds bd;
  bd.init(lv, start, L, active);
  // refinement: x of the row above the current one (the previous block's
  // last row before the block's first row)
  Tin xup = Tin{};
  if constexpr (kRef) {
    if (active && start > 0) xup = rf.x[start - 1];
  }

  // virtual state before row 1 (relation x_0 = f): rbeta = 1, c_prev = 0,
  // g = 0, alpha = -1; first interior unknown x_1 = P - Q f - S x_1 with
  // P = Q = 0, S = -1.
  T rbp = Ar::one(), cprev = Ar::zero(), g = Ar::zero(), al = Ar::neg(Ar::one());
  T P = Ar::zero(), Q = Ar::zero(), S = Ar::neg(Ar::one());
  T a0 = Ar::zero(), b0 = Ar::one(), c0 = Ar::zero(), d0 = Ar::zero();
  T beta = Ar::one(), clast = Ar::zero();
  bool bad = false;
  // range of the rows (fp64 inputs in narrower arithmetic), and the packed
  // system the current row belongs to (for its |d / b| code)
  RowChk chk;
  int64_t sys = lv.nbnd > 0 && active ? bd.first : 0;

  // The first interior unknown's chain (P, Q, S) only adds terms scaled by
  // S, whose magnitude falls by |c / beta| < 1 every row of a strictly
  // diagonally dominant block.  Where the policy allows (Ar::kSkipChain),
  // once every lane's |S| is below 2^-60 the rest of the chain is below
  // rounding and the rows skip it (kChain false); they check |c| <= |beta|
  // instead, so S cannot grow back, and a block where that fails reports a
  // pivot failure (not dominant).
  bool chain = true, nondom = false;

  // one interior row (1 <= row <= L-2).  The product chains alpha and S and
  // the accumulators P and Q are left unnormalised here and renormalised
  // once per chunk (renorm), which bounds their low parts to a few ulps.
  auto interior = [&](const T av, const T bv, const T cv, const T dv, auto kChain) {
    const T ratio = Ar::mul_nn(av, rbp);
    beta = Ar::sub_mul_dom(bv, ratio, cprev);
    g = Ar::sub_mul(dv, ratio, g);
    al = Ar::mul_neg_nn(ratio, al);
    bad |= Ar::bad_pivot(beta);
    const T rbeta = Ar::rcp(beta);
    if constexpr (decltype(kChain)::value) {
      const T tt = Ar::mul_nn(S, rbeta);
      P = Ar::sub_mul_nn(P, tt, g);
      Q = Ar::sub_mul_nn(Q, tt, al);
      S = Ar::mul_neg_nn(tt, cv);
    } else {
      nondom |= !Ar::mag_le(cv, beta);
    }
    rbp = rbeta;
    cprev = cv;
  };
  auto renorm = [&]() {
    al = Ar::norm(al);
    S = Ar::norm(S);
    P = Ar::norm(P);
    Q = Ar::norm(Q);
  };
  // checkpoint after row `row` (a multiple of K minus one), when the next K
  // rows start with an interior row (Stage 3 restarts its chunk there)
  auto checkpoint = [&](int row) {
    if (active && row + 1 <= L - 2) {
      const int64_t slot = (int64_t)((row + 1) / K - 1) * lv.p + k;
      Ar::to(ck_gam[slot], Ar::mul(cprev, rbp));
      Ar::to(ck_y[slot], Ar::mul(Ar::norm(g), rbp));
      Ar::to(ck_v[slot], Ar::mul(Ar::norm(al), rbp));
    }
  };

  for (int ch = 0; ch < nch; ++ch) {
    const int row0 = ch * R;
    fetch(ch + kS1Stages - 1);
    cp_async_wait<kS1Stages - 1>();
    __syncwarp();
    Tin* const tb = tile + (ch % kS1Stages) * TL::kBuf;
    Tin* const t = tb + lane * TL::kStride;
    const bool clean = !__any_sync(0xffffffffu, bd.cnt > 0 && bd.touches(start + row0, R));
    const int kind = chunk_kind(ch, row0, R, lmin, luni, clean);
    // one unrolled body for the three kinds (only row 0 and row R-1 test,
    // warp-uniformly, whether they are the block's f or l row), compiled
    // with and without the first unknown's chain
    auto fast_chunk = [&](auto kChain) {
      const bool first = kind == kFirst, last = kind == kLast;
#pragma unroll
      for (int r = 0; r < R; r += V) {
        const Vec16<Tin> xa = lds16(t + r), xb = lds16(t + TL::kArr + r),
                         xc = lds16(t + 2 * TL::kArr + r), xd = lds16(t + 3 * TL::kArr + r);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int rr = r + v;
          // a of the system's first row and c of its last are never read
          const bool cut_c = rr == R - 1 && last && k == lv.p - 1;
          const Tin ain = (rr == 0 && first && k == 0) ? Tin{} : xa.v[v];
          const Tin cin = cut_c ? Tin{} : xc.v[v];
          Tin din = xd.v[v];
          if constexpr (kRef) {  // the residual of the current x
            const Tin x0 = t[4 * TL::kArr + rr];
            din = residual_row(ain, xb.v[v], cin, din, xup, x0,
                               cut_c ? Tin{} : t[4 * TL::kArr + rr + 1]);
            xup = x0;
            t[3 * TL::kArr + rr] = din;
          }
          T av, bv, cv, dv;
          Ar::template row<true>(ain, xb.v[v], cin, din, av, bv, cv, dv, chk);
          if (rr == 0 && first) {  // the block's first row: f's equation
            a0 = av; b0 = bv; c0 = cv; d0 = dv;
          } else if (rr == R - 1 && last) {  // the block's last row
            const T ratio = Ar::mul_nn(av, rbp);
            beta = Ar::sub_mul_dom(bv, ratio, cprev);
            g = Ar::sub_mul(dv, ratio, g);
            al = Ar::mul_neg_nn(ratio, al);
            clast = cv;
          } else {
            interior(av, bv, cv, dv, kChain);
            if constexpr (R > K) {  // chunk spans several checkpoint intervals
              if ((rr + 1) % K == 0 && rr + 1 < R) checkpoint(row0 + rr);
            }
          }
        }
      }
    };
    if (kind != kSlow) {
      if constexpr (Ar::kSkipChain) {
        if (chain) fast_chunk(std::true_type{});
        else fast_chunk(std::false_type{});
      } else {
        fast_chunk(std::true_type{});
      }
    } else {
#pragma unroll 1
      for (int r = 0; r < R; ++r) {
        const int row = row0 + r;
        if (row < L) {
          // couplings cut at system boundaries (and a[0], c[n-1]) are never read
          bool cut_a = k == 0 && row == 0, cut_c = k == lv.p - 1 && row == L - 1;
          if (bd.cnt > 0) {
            if (bd.is(start + row)) {  // a new packed system starts here
              cut_a = true;
              if (lv.dmax) codes_raise(lv.dmax, sys, chk.dcode(), chk.ecode, chk.fcode());
              chk.reset_codes();
              ++sys;
            }
            cut_c |= bd.is(start + row + 1);
          }
          Tin din = t[3 * TL::kArr + r];
          if constexpr (kRef) {
            const Tin x0 = t[4 * TL::kArr + r];
            din = residual_row(cut_a ? Tin{} : t[r], t[TL::kArr + r],
                               cut_c ? Tin{} : t[2 * TL::kArr + r], din, cut_a ? Tin{} : xup, x0,
                               cut_c ? Tin{} : t[4 * TL::kArr + r + 1]);
            xup = x0;
            t[3 * TL::kArr + r] = din;
          }
          T av, bv, cv, dv;
          Ar::template row<true>(cut_a ? Tin{} : t[r], t[TL::kArr + r],
                                 cut_c ? Tin{} : t[2 * TL::kArr + r], din, av, bv, cv, dv, chk);
          if (row == 0) {
            a0 = av; b0 = bv; c0 = cv; d0 = dv;
          } else if (row < L - 1) {
            if (!Ar::kSkipChain || chain) interior(av, bv, cv, dv, std::true_type{});
            else interior(av, bv, cv, dv, std::false_type{});
            if constexpr (R > K) {
              if ((row + 1) % K == 0 && r + 1 < R) checkpoint(row);
            }
          } else {
            const T ratio = Ar::mul_nn(av, rbp);
            beta = Ar::sub_mul_dom(bv, ratio, cprev);
            g = Ar::sub_mul(dv, ratio, g);
            al = Ar::mul_neg_nn(ratio, al);
            clast = cv;
          }
        }
      }
    }
    renorm();
    // the checkpoint at the chunk's end (row0 + R is a multiple of K when
    // K divides R, and every K / R chunks otherwise)
    if (((row0 + R) % K) == 0) checkpoint(row0 + R - 1);
    if constexpr (Ar::kSkipChain) {
      if (chain && __all_sync(0xffffffffu, !active || Ar::chain_small(S))) chain = false;
    }
    if constexpr (kRef) {  // the chunk's residual (in the d slots) out
      __syncwarp();
      store_chunk<Tin, R, kVec16>(rf.r, tb + 3 * TL::kArr, pm, row0);
    }
    __syncwarp();  // the buffer is refilled by the next iteration's copies
  }
  bad |= nondom;
  if (active) {
    bad |= Ar::bad_pivot(beta);
    if (L == 1) {
      // a one-row block is a one-row system (tails are merged otherwise):
      // b0 f = d0, and a decoupled identity row for the unused l
      Ar::to(ra[2 * k], Ar::zero());
      Ar::to(rb[2 * k], b0);
      Ar::to(rc[2 * k], Ar::zero());
      Ar::to(rd[2 * k], d0);
      Ar::to(ra[2 * k + 1], Ar::zero());
      Ar::to(rb[2 * k + 1], Ar::one());
      Ar::to(rc[2 * k + 1], Ar::zero());
      Ar::to(rd[2 * k + 1], Ar::zero());
    } else {
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
    }
    if (bad || chk.b_bad()) atomicOr(status, ST_BAD_PIVOT);
    if (chk.range_bad()) atomicOr(status, ST_RANGE);
  }
  if (lv.dmax) codes_raise_warp(lv.dmax, sys, active, chk);
}

// ------------------------------------------------------------------ Stage 3
// kRef: a refinement step (RefineIO): d is the residual Stage 1 wrote, the
// result is added to x in place and the maxima go to rf.max2.
template <class Ar, class Tin, class Tred, int R, int W, bool kVec16, bool kRef = false>
__global__ void __launch_bounds__(W * 32)
    k_stage3(Level lv, const Tin* __restrict__ a, const Tin* __restrict__ b,
             const Tin* __restrict__ c, const Tin* __restrict__ d, const Tred* __restrict__ xred,
             const Tred* __restrict__ ck_gam, const Tred* __restrict__ ck_y,
             const Tred* __restrict__ ck_v, Tin* __restrict__ x, int* __restrict__ status,
             RefineIO rf = {}) {
  using T = typename Ar::T;
  using TL = Tile<Tin, R, kRef ? 5 : 4>;
  using TL3 = Tile3<Tin, Tred, R, kRef ? 5 : 4>;
  static_assert(!kRef || std::is_same<Tin, double>::value, "refinement steps are fp64");
  constexpr int V = TL::kVec;
  static_assert(sizeof(T) <= sizeof(Tin), "boundary chunks park T values in Tin slots");
  static_assert(sizeof(Tred) == 4 || sizeof(Tred) == 8, "checkpoint element size");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // CTAs run in the reverse of Stage 1's order: the rows Stage 1 read last
  // are the ones still in L2 (and the next solve's Stage 1 starts on the
  // rows this one read last)
  const int64_t k0 = lv.k_begin + ((int64_t)(gridDim.x - 1 - blockIdx.x) * W + warp) * 32;
  if (k0 >= lv.k_end) return;
  const int nb = (int)(lv.k_end - k0 < 32 ? lv.k_end - k0 : 32);
  const int64_t k = k0 + lane;
  const bool active = lane < nb;
  const int L = active ? block_len(lv, k) : 0;
  const int nch = warp_chunks(lv, k0, nb, R);
  const int lmin = warp_lmin(lv, k0, nb);
  const int luni = warp_luni(lv, k0, nb);

  unsigned char* wbase = smem_raw + warp * TL3::kBytesPerWarp;
  Tin* tile = reinterpret_cast<Tin*>(wbase);
  Tred* ckbuf = reinterpret_cast<Tred*>(wbase + TL::kBytesPerWarp);  // [buf][3][32]
  const Tin* const srcs[4] = {a, b, c, d};
  const Tin* const xsrc[1] = {x};  // refinement: the current iterate, a fifth array
  PieceMap<Tin, R> pm;
  pm.init(lv, k0, nb, lane);
  // the lane's checkpoint for chunk ch (written by Stage 1 after row ch*R-1)
  auto load_ck = [&](Tred* dst, int ch) {
    if (active && ch > 0 && ch * R <= L - 2) {
      const int64_t slot = (int64_t)(ch - 1) * lv.p + k;
      cp_async<sizeof(Tred)>(dst + lane, ck_gam + slot);
      cp_async<sizeof(Tred)>(dst + 32 + lane, ck_y + slot);
      cp_async<sizeof(Tred)>(dst + 64 + lane, ck_v + slot);
    }
  };
  load_chunk<Tin, R, kVec16>(tile, srcs, 4, pm, (nch - 1) * R);
  if constexpr (kRef) load_chunk<Tin, R, kVec16>(tile + 4 * TL::kArr, xsrc, 1, pm, (nch - 1) * R);
  load_ck(ckbuf, nch - 1);
  cp_async_commit();
  unsigned long long mdel = 0, mx = 0;  // refinement maxima (bit patterns)

  const int64_t start = k * (int64_t)lv.m;
  Bounds bd;
  bd.init(lv, start, L, active);
  T f = Ar::zero(), l = Ar::zero();
  if (active) {
    f = Ar::from(xred[2 * k]);
    l = Ar::from(xred[2 * k + 1]);
  }
  T xnext = l;  // x of the row below the chunk being processed
  bool bad = false, oob = false;
  RowChk nochk;  // the rows' range was checked by Stage 1

  // chunks bottom-up: ch = nch-1 .. 0; buffer parity follows the visiting order
  for (int it = 0; it < nch; ++it) {
    const int ch = nch - 1 - it;
    const int row0 = ch * R;
    if (ch > 0) {
      load_chunk<Tin, R, kVec16>(tile + ((it + 1) & 1) * TL::kBuf, srcs, 4, pm, row0 - R);
      if constexpr (kRef)
        load_chunk<Tin, R, kVec16>(tile + ((it + 1) & 1) * TL::kBuf + 4 * TL::kArr, xsrc, 1, pm,
                                   row0 - R);
      load_ck(ckbuf + ((it + 1) & 1) * 96, ch - 1);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    Tin* tb = tile + (it & 1) * TL::kBuf;
    Tin* t = tb + lane * TL::kStride;

    // relation entering the chunk: x_{row0-1} = zp - gp * x_{row0}
    T zp = f, gp = Ar::zero();
    if (active && ch > 0 && row0 <= L - 2) {
      const Tred* ck = ckbuf + (it & 1) * 96;
      gp = Ar::from(ck[lane]);
      zp = Ar::sub_mul(Ar::from(ck[32 + lane]), Ar::from(ck[64 + lane]), f);
    }
    const bool clean = !__any_sync(0xffffffffu, bd.cnt > 0 && bd.touches(start + row0, R));
    const int kind = chunk_kind(ch, row0, R, lmin, luni, clean);
    if (kind != kSlow) {
      // unrolled chunk: forward over the interior rows, back-substitution
      // from the row below; only row 0 (kFirst: f) and row R-1 (kLast: l)
      // test their role, warp-uniformly
      const bool first = kind == kFirst, last = kind == kLast;
      T Z[R], G[R];
      Tin xo[R];
#pragma unroll
      for (int r = 0; r < R; r += V) {
        const Vec16<Tin> xa = lds16(t + r), xb = lds16(t + TL::kArr + r),
                         xc = lds16(t + 2 * TL::kArr + r), xd = lds16(t + 3 * TL::kArr + r);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int rr = r + v;
          if ((rr == 0 && first) || (rr == R - 1 && last)) continue;
          T av, bv, cv, dv;
          Ar::template row<false>(xa.v[v], xb.v[v], xc.v[v], xd.v[v], av, bv, cv, dv, nochk);
          const T beta = Ar::sub_mul_dom(bv, av, gp);
          bad |= Ar::bad_pivot(beta);
          const T rbeta = Ar::rcp(beta);
          zp = Ar::mul_nn(Ar::sub_mul(dv, av, zp), rbeta);
          gp = Ar::mul_nn(cv, rbeta);
          Z[rr] = zp;
          G[rr] = gp;
        }
      }
      // back-substitution (x over the Z slots), then the output conversion
#pragma unroll
      for (int r = R - 1; r >= 0; --r) {
        if (r == R - 1 && last) {
          Z[r] = l;  // xnext is l already
        } else if (r == 0 && first) {
          Z[r] = f;
        } else {
          xnext = Ar::sub_mul(Z[r], G[r], xnext);
          Z[r] = xnext;
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        Ar::to(xo[r], Z[r]);
        oob |= Ar::out_bad(xo[r]);
        if constexpr (kRef) {  // x += delta (lanes past the level's last block: no rows)
          const Tin xn = t[4 * TL::kArr + r] + xo[r];
          if (active) {
            mdel = max(mdel, abs_bits(xo[r]));
            mx = max(mx, abs_bits(xn));
          }
          xo[r] = xn;
        }
      }
#pragma unroll
      for (int r = 0; r < R; r += V) {
        Vec16<Tin> w;
#pragma unroll
        for (int v = 0; v < V; ++v) w.v[v] = xo[r + v];
        *reinterpret_cast<float4*>(t + r) = *reinterpret_cast<const float4*>(&w);
      }
    } else {
      // boundary chunk: the same recurrences, row by row, with the pivots and
      // right-hand sides parked in the lane's b and c slots
      T* zs = reinterpret_cast<T*>(t + TL::kArr);
      T* gs = reinterpret_cast<T*>(t + 2 * TL::kArr);
#pragma unroll 1
      for (int r = 0; r < R; ++r) {
        const int row = row0 + r;
        if (row >= 1 && row <= L - 2) {
          T av, bv, cv, dv;
          Ar::template row<false>(t[r], t[TL::kArr + r], t[2 * TL::kArr + r],
                                  t[3 * TL::kArr + r], av, bv, cv, dv, nochk);
          if (bd.cnt > 0) {  // couplings cut at system boundaries
            if (bd.is(start + row)) av = Ar::zero();
            if (bd.is(start + row + 1)) cv = Ar::zero();
          }
          const T beta = Ar::sub_mul_dom(bv, av, gp);
          bad |= Ar::bad_pivot(beta);
          const T rbeta = Ar::rcp(beta);
          zp = Ar::mul_nn(Ar::sub_mul(dv, av, zp), rbeta);
          gp = Ar::mul_nn(cv, rbeta);
          zs[r] = zp;
          gs[r] = gp;
        }
      }
#pragma unroll 1
      for (int r = R - 1; r >= 0; --r) {
        const int row = row0 + r;
        if (row < L) {
          T xr;
          if (row == 0) {
            xr = f;
          } else if (row == L - 1) {
            xr = l;
          } else {
            xr = Ar::sub_mul(zs[r], gs[r], xnext);
            xnext = xr;
          }
          Ar::to(t[r], xr);
          oob |= Ar::out_bad(t[r]);
          if constexpr (kRef) {  // x += delta
            const Tin xn = t[4 * TL::kArr + r] + t[r];
            mdel = max(mdel, abs_bits(t[r]));
            mx = max(mx, abs_bits(xn));
            t[r] = xn;
          }
        }
      }
    }
    // the chunk's x is in the lanes' a slots (a is no longer needed): out
    __syncwarp();
    store_chunk<Tin, R, kVec16>(x, tb, pm, row0);
    __syncwarp();  // the buffer is refilled by the next iteration's copies
  }
  if (active && bad) atomicOr(status, ST_BAD_PIVOT);
  if (active && oob) atomicOr(status, ST_RANGE);
  if constexpr (kRef) {
    for (int o = 16; o > 0; o >>= 1) {
      mdel = max(mdel, __shfl_xor_sync(0xffffffffu, mdel, o));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    // most warps see maxima already raised past theirs: read before the atomic
    if (lane == 0) {
      if (mdel > *(volatile unsigned long long*)&rf.max2[0]) atomicMax(&rf.max2[0], mdel);
      if (mx > *(volatile unsigned long long*)&rf.max2[1]) atomicMax(&rf.max2[1], mx);
    }
  }
}

// ------------------------------------------------------------------ small systems
// One warp solves a system of n <= 64 rows by parallel cyclic reduction
// (Hockney 1965): at stride s every row eliminates its neighbours at
// distance s, after ceil(log2 n) steps each row is decoupled and
// x_i = d_i / b_i.  Rows outside [0, n) act as identity rows.
constexpr int kBaseMax = 64;

// dmax (level 0 of fp64 inputs in narrower arithmetic, else null): the
// per-system range codes, raised here; x is checked for range.
template <class Ar, class Tin, class Tout>
__global__ void __launch_bounds__(32)
    k_base(int64_t n, const Tin* __restrict__ a, const Tin* __restrict__ b,
           const Tin* __restrict__ c, const Tin* __restrict__ d, Tout* __restrict__ x,
           const int64_t* __restrict__ bnd, int64_t nbnd, int* __restrict__ status,
           unsigned* __restrict__ dmax) {
  using T = typename Ar::T;
  __shared__ T sa[kBaseMax], sb[kBaseMax], sc[kBaseMax], sd[kBaseMax];
  const int lane = threadIdx.x;
  const int nn = (int)n;
  bool bad = false, oob = false;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    if (i < nn) {
      bool start = (i == 0), end = (i == nn - 1);
      int64_t sys = 0;
      for (int64_t j = 0; j < nbnd; ++j) {  // packed systems: cut the couplings
        start |= bnd[j] == i;
        end |= bnd[j] == i + 1;
        sys += bnd[j] <= i;
      }
      RowChk rc;
      Ar::template row<true>(start ? Tin{} : a[i], b[i], end ? Tin{} : c[i], d[i], sa[i], sb[i],
                             sc[i], sd[i], rc);
      oob |= rc.range_bad();
      bad |= rc.b_bad();
      if (dmax) codes_raise(dmax, sys, rc.dcode(), rc.ecode, rc.fcode());
    } else {
      sa[i] = Ar::zero(); sb[i] = Ar::one(); sc[i] = Ar::zero(); sd[i] = Ar::zero();
    }
  }
  __syncwarp();
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
      Tout xv;
      Ar::to(xv, Ar::mul(sd[i], Ar::rcp(sb[i])));
      oob |= Ar::out_bad(xv);
      x[i] = xv;
    }
  }
  if (bad) atomicOr(status, ST_BAD_PIVOT);
  if (oob) atomicOr(status, ST_RANGE);
}

}  // namespace tps
