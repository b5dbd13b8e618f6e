// Host-side internals of libtps: the plan object, the level geometry of the
// recursive partition solve, and the launch entry points of each
// translation unit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/tps.h"
#include "partition_kernels.cuh"

namespace tps {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Rows per shared-memory chunk (and checkpoint spacing) for an element size.
#ifndef TPS_CHUNK_ROWS_8B
#define TPS_CHUNK_ROWS_8B 8  // Stage-3 chunk rows (checkpoint spacing) for 8-byte elements
#endif
inline int chunk_rows(size_t elem_bytes) { return elem_bytes >= 8 ? TPS_CHUNK_ROWS_8B : 16; }
template <class T>
constexpr int kChunkRows = sizeof(T) >= 8 ? TPS_CHUNK_ROWS_8B : 16;
#ifndef TPS_WARPS_PER_CTA
#define TPS_WARPS_PER_CTA 1
#endif
constexpr int kWarpsPerCta = TPS_WARPS_PER_CTA;
// devices a process may use (per-device caches of kernel attributes)
constexpr int kMaxDevices = 64;

// One level of the recursive solve: the system at this level has lv.n rows
// and is split into lv.p blocks; its reduced system (2 lv.p rows) and the
// Stage-1 checkpoints live in the workspace at the given offsets.
struct LevelPlan {
  Level lv;
  int R;
  size_t off_red[5];  // ra, rb, rc, rd, xr
  size_t off_ck[3];   // gamma, y, v
};

// Block geometry for n rows and nominal block length m (m >= 2, n > m is
// not required): p = ceil(n/m) blocks, a one-row tail merged into the block
// before it so every block has >= 2 rows.
// Argument checks shared by the entry points: managed memory or device
// memory of `device`, aligned to `align`; the plan's device is current.
bool device_ptr_ok(const void* p, size_t align, int device);
bool on_plan_device(const tps_plan_s* P);

Level make_level(int64_t n, int m, int R);

// Levels of the recursive solve of an n-row system (empty when n fits the
// one-warp base solve), with workspace offsets starting at `base`; returns
// the end offset.
size_t build_levels(int64_t n, int m0, int mr, size_t top_elem, size_t red_elem, size_t base,
                    std::vector<LevelPlan>& out);

struct HostPipe;  // streams and events of tps_solve_host_async

}  // namespace tps

struct tps_plan_s {
  tps_plan_desc desc;
  int32_t device = -1;  // the device current at tps_plan; every call must use it
  int32_t m = 0, m_reduced = 0, streams = 1;
  int64_t chunk = 0;
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0, ws_needed = 0;
  bool ws_owned = false;
  int* d_status = nullptr;     // device status word (first bytes of ws)
  // per-system range codes of the last solve's rows (double-float plans and
  // the first fp32 solve of a mixed one; kCodes x max(1, batch_max) words
  // after the header), zero between solves
  size_t off_dmax = 0;
  // the mixed solve's corrections (right-hand sides small by construction)
  // skip the range codes
  bool codes_off = false;
  double* d_scalars = nullptr; // refinement reductions (next bytes of ws)
  size_t off_levels = 0;       // first level buffer offset
  size_t off_refine = 0;       // refinement residual and correction vectors
  cudaStream_t last_stream = nullptr;
  int32_t last_levels = 0;
  int32_t last_iters = 0;
  double last_corr = 0.0;
  float stage_ms[4] = {0, 0, 0, 0};
  int32_t host_status = 0;     // numeric status found on the host (refinement)
  tps::HostPipe* pipe = nullptr;
  // TPS_TRACE: a ring of 4 events per solve (before/after Stage 1, after
  // Stage 2, after Stage 3 of level 0), averaged by tps_plan_query
  cudaEvent_t* trace_ev = nullptr;
  int32_t trace_slots = 0;
  int64_t trace_count = 0;
  // TPS_GRAPH: the captured solve and the arguments it was captured with
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;
  int64_t gkey[12] = {};
  // TPS_GRAPH without TPS_TRACE: the whole solve, captured once per
  // geometry and set of pointers, replayed as one graph launch
  cudaGraphExec_t solve_graph = nullptr;
  int64_t sgkey[16] = {};
  int32_t sg_onchip = 0, sg_levels = 0;
  // TPS_ZERO_COPY: the device can read and write pageable host memory
  bool pageable_ok = false;
  // one-warp windowed solve (TPS_TRUNCATE): its relation buffer
  size_t off_rel = 0;
  // on-chip solve: exchange rows for the CTAs' interface equations, and
  // which part of the last solve ran on chip (0 none, 1 all, 2 reduced)
  size_t off_xch = 0;
  int32_t last_onchip = 0;
  int32_t graph_onchip = 0;  // last_onchip and last_levels of the captured Stage 2
  int32_t graph_levels = 0;
  // test hook (TPS_TEST_ONCHIP_TIMEOUT=1 at plan creation): the on-chip
  // solve's grid barrier waits for one CTA more than it launches, so the
  // bounded wait runs out and the solve reports TPS_ERR_TIMEOUT
  bool test_barrier_extra = false;
  bool test_unfused_refine = false;  // TPS_TEST_UNFUSED_REFINE=1 at plan time
  int32_t last_refine_fused = 0;     // the last mixed solve used refine_step
  // batched work list (device) and its capacity in entries
  void* d_work = nullptr;
  size_t work_cap = 0;
  // TPS_HOST_OVERLAP: the twin plan (second buffer set and streams) that
  // takes every other system of tps_solve_host_many_async, one stream per
  // buffer set through which that set's systems are ordered, and events to
  // fork from and join back into the caller's stream
  tps_plan_s* twin = nullptr;
  cudaStream_t lane[2] = {nullptr, nullptr};
  cudaEvent_t lane_ev[3] = {nullptr, nullptr, nullptr};
};

namespace tps {

// Enqueue the recursive partition solve of one device-resident system.
// dtype selects the arithmetic; a..x are device pointers of the I/O type.
// ev (optional, 4 events) is recorded before Stage 1, after Stage 1, after
// Stage 2 and after Stage 3 of level 0.
// bnd/nbnd: for packed systems, the first rows of systems 1.. (device,
// sorted); the couplings there are cut.  lv[0].lv must carry the same.
tps_status run_solve(tps_plan_s* P, int64_t n, const void* a, const void* b, const void* c,
                     const void* d, void* x, cudaStream_t s, const std::vector<LevelPlan>& lv,
                     cudaEvent_t* ev, const int64_t* bnd = nullptr, int64_t nbnd = 0);

// Level-0 pieces of the solve for the chunked host pipeline: Stage 1 and
// Stage 3 on blocks [kb, ke), Stage 2 on the whole reduced system, and the
// one-warp solve for n <= kBaseMax.
cudaError_t stage1_range(tps_plan_s* P, const LevelPlan& L, int64_t kb, int64_t ke,
                         const void* a, const void* b, const void* c, const void* d,
                         cudaStream_t s);
cudaError_t stage3_range(tps_plan_s* P, const LevelPlan& L, int64_t kb, int64_t ke,
                         const void* a, const void* b, const void* c, const void* d, void* x,
                         cudaStream_t s);
cudaError_t reduced_solve(tps_plan_s* P, const std::vector<LevelPlan>& levels, cudaStream_t s);
// One correction step of the mixed solve fused into level 0's sweeps
// (levels non-empty): r = d - A x (fp64) formed in Stage 1, the fp32 solve
// of A delta = r, x += delta in Stage 3; max2 (two device words, zeroed
// here) receives max |delta| and max |x| as non-negative double bit
// patterns.  r: n doubles of scratch.
cudaError_t refine_step(tps_plan_s* P, const std::vector<LevelPlan>& levels, const double* a,
                        const double* b, const double* c, const double* d, double* x, double* r,
                        unsigned long long* max2, cudaStream_t s);
// Bytes of the on-chip solve's exchange rows (part of every plan workspace).
size_t onchip_exchange_bytes();
// The single-launch on-chip solve of one system if it fits on this device
// (used = true), else nothing.  xch: onchip_exchange_bytes() of device
// memory; bar: a device counter (zeroed by the call); status: the device
// status word; dmax: for double-float, one system's kCodes range codes,
// zero before the launch and left zero after it (else null).
cudaError_t onchip_solve(int dtype, int64_t n, const void* a, const void* b, const void* c,
                         const void* d, void* x, void* xch, unsigned* bar, int* status,
                         cudaStream_t s, bool& used, unsigned* dmax);
// TPS_TRUNCATE: the windowed solve of one device-resident system.
tps_status run_truncated(tps_plan_s* P, int64_t n, const void* a, const void* b, const void* c,
                         const void* d, void* x, cudaStream_t s);
// Largest extended window (kept rows + both halos) of the one-CTA windowed
// solve.
int truncate_rows_max();
// Rows per lane block of the one-warp windowed solve for R kept rows and h
// halo rows (R + 2 h = 32 mb), or 0 when that solve does not apply.
int truncate_warp_mb(int R, int h);
// Bytes of the one-warp windowed solve's relation buffer for n_max rows.
size_t truncate_rel_bytes(int64_t n_max, int R, int h, int dtype);
// Copy `bytes` between host and device memory with a streaming kernel (SM
// loads and stores, no copy engine); either side may be host memory the
// device can address.  bytes and both pointers: multiples of 4.
cudaError_t kernel_copy(void* dst, const void* src, size_t bytes, cudaStream_t s);
// The same, captured once into a CUDA graph (TPS_GRAPH) and replayed.
cudaError_t reduced_solve_graph(tps_plan_s* P, const std::vector<LevelPlan>& levels,
                                cudaStream_t s);
cudaError_t base_solve(tps_plan_s* P, int64_t n, const void* a, const void* b, const void* c,
                       const void* d, void* x, cudaStream_t s, const int64_t* bnd = nullptr,
                       int64_t nbnd = 0);
// The per-system range codes that level 0 of this plan's solves raises
// (null where the arithmetic needs no such test).
unsigned* level0_dmax(tps_plan_s* P);
// After level 0 has loaded every row: flag ST_RANGE for each of `count`
// systems whose range codes are out of range, and clear the codes.
cudaError_t dcode_check(tps_plan_s* P, int64_t count, cudaStream_t s);

// Mixed-precision refinement of one device-resident system (or packed
// systems): fp32 partition elimination, fp64 residual and update.  Reads two
// maxima back to the host after every correction (synchronises `s`).
tps_status run_refine(tps_plan_s* P, int64_t n, const double* a, const double* b,
                      const double* c, const double* d, double* x, cudaStream_t s,
                      const std::vector<LevelPlan>& lv, const int64_t* bnd, int64_t nbnd);

size_t elem_bytes_io(int dtype);
size_t elem_bytes_red(int dtype);

}  // namespace tps
