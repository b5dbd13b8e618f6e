/*
 * tps.h -- C ABI of libtps, a GB300 (sm_103a) solver for tridiagonal systems
 * by the partition method.
 *
 * The method (paper Sec. 1, citing Austin et al. 2004; Sec. 2.2) splits the
 * n x n tridiagonal matrix into blocks of m consecutive rows and solves
 *   Stage 1  per block: eliminate the interior rows, leaving two equations
 *            in the block's first and last unknown (its interface unknowns);
 *   Stage 2  the reduced tridiagonal system in all interface unknowns;
 *   Stage 3  per block: recover the interior unknowns from the interface
 *            values.
 * Here all three stages run on the GPU; Stage 2 applies the same method
 * recursively until the reduced system fits in shared memory (one
 * cooperative launch finishes it) or in one warp (parallel cyclic
 * reduction).  The
 * host-resident pipeline (Sec. 2.2, Eq. 2) overlaps chunked host-to-device
 * copies, kernels and device-to-host copies on S CUDA streams, S a power of
 * two up to 32 (Sec. 2.1).
 *
 * Conventions shared by every entry point
 *   Row i reads  a[i]*x[i-1] + b[i]*x[i] + c[i]*x[i+1] = d[i].  a[0] and
 *   c[n-1] (per system in a batch) are never used, so packed systems never
 *   couple.  Arrays are contiguous, one element per row, of the plan's I/O
 *   type (double for TPS_F64, TPS_F64_DF and TPS_MIXED_F32_F64; float for
 *   TPS_F32).  The caller owns every array; inputs are not modified; x must
 *   not overlap an input.  The matrix should be strictly diagonally
 *   dominant (no pivoting is done); a zero or non-finite pivot is reported
 *   through tps_plan_query, not by the return value.
 *   Calls are stream-ordered and asynchronous: argument and launch errors
 *   come back as the return value, numeric errors (TPS_ERR_ZERO_PIVOT,
 *   TPS_ERR_RANGE, TPS_ERR_NO_CONVERGENCE) from tps_plan_query after the
 *   stream has been synchronised.  A plan may be used by one stream at a
 *   time.
 *   A plan belongs to the device that is current when tps_plan creates it:
 *   every later call on it needs that device current, and its device
 *   arrays on that device (or managed), else TPS_ERR_INVALID_ARG.  Distinct
 *   plans may be used from different host threads at the same time; one
 *   plan by one thread at a time.
 *   `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 */
#ifndef TPS_H
#define TPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TPS_OK = 0,
  TPS_ERR_INVALID_ARG = 1,    /* bad pointer, size, alias, or plan misuse      */
  TPS_ERR_UNSUPPORTED = 2,    /* valid request this library does not serve     */
  TPS_ERR_CUDA = 3,           /* a CUDA runtime call failed                    */
  TPS_ERR_OOM = 4,            /* device or pinned allocation failed            */
  TPS_ERR_ZERO_PIVOT = 5,     /* zero/non-finite pivot met (matrix not SDD)    */
  TPS_ERR_NO_CONVERGENCE = 6, /* mixed-precision refinement did not converge   */
  TPS_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up            */
  TPS_ERR_RANGE = 8           /* an input or x outside what the arithmetic     */
                              /* represents (see TPS_F64_DF)                   */
} tps_status;

typedef enum {
  TPS_F64 = 0,           /* fp64 I/O, native fp64 arithmetic (the plain solve)  */
  TPS_F32 = 1,           /* fp32 I/O and arithmetic                             */
  TPS_MIXED_F32_F64 = 2, /* fp64 I/O; fp32 elimination, fp64 residual/update,   */
                         /* iterative refinement to the plan's tolerance        */
  TPS_F64_DF = 3         /* fp64 I/O; double-float arithmetic (pairs of fp32)   */
                         /* on the fp32 pipes, about 2^-46 relative per op.     */
                         /* Each row is scaled exactly by the power of two that */
                         /* brings b[i] into [1, 2), so any fp64 scaling of the */
                         /* rows is served (x unchanged).  The pairs hold x at  */
                         /* full precision while max |d[i] / b[i]| lies in      */
                         /* [2^-84, 2^84].  Reported after the solve            */
                         /* (tps_plan_query): TPS_ERR_ZERO_PIVOT for a b[i]     */
                         /* that is 0, subnormal, infinite or NaN;              */
                         /* TPS_ERR_RANGE for an a[i], c[i] or d[i] above        */
                         /* 2^84 |b[i]| (or not finite), for a system whose     */
                         /* |d[i] / b[i]| is below 2^-84 in every row with      */
                         /* d[i] != 0, for an entry taken as 0 (a[i], c[i]      */
                         /* below 2^-103 |b[i]|, d[i] below 2^-129 |b[i]|) in a */
                         /* row whose |b[i]| is so large against the system    */
                         /* that the residual could suffer, and for an x at or  */
                         /* above 2^101.  TPS_F64 has none of these limits.     */
} tps_dtype;

typedef enum {
  TPS_DEVICE = 0,     /* arrays in device memory (tps_solve, tps_solve_batched) */
  TPS_HOST_PINNED = 1 /* arrays in pinned host memory (tps_solve_host_async)    */
} tps_residency;

/* tps_plan_desc.flags */
#define TPS_TUNE_PREDICT 1u       /* fill zero m/streams/chunk from the predictor */
#define TPS_TUNE_EXHAUSTIVE 2u    /* time the candidate grid on the device        */
#define TPS_TRACE 4u              /* record per-stage event times (tps_plan_query) */
#define TPS_EXTERNAL_WORKSPACE 8u /* caller supplies the workspace                */
#define TPS_GRAPH 16u             /* replay the solve as one CUDA graph launch    */
#define TPS_ZERO_COPY 32u         /* host residency: kernels, not copy engines,   */
                                  /* move host data (see tps_solve_host_async)    */
#define TPS_NO_ONCHIP 64u         /* never use the single-launch on-chip solve    */
#define TPS_TRUNCATE 128u         /* approximate windowed solve (see tps_solve)   */
#define TPS_HOST_OVERLAP 256u     /* host residency: a second buffer set so that  */
                                  /* tps_solve_host_many_async overlaps systems   */

typedef struct {
  int64_t n_max;     /* largest n of tps_solve / tps_solve_host_async, or the  */
                     /* largest total row count of tps_solve_batched           */
  int64_t batch_max; /* largest system count of tps_solve_batched (0: none)    */
  int32_t dtype;     /* tps_dtype                                              */
  int32_t residency; /* tps_residency (informs the predictor)                  */
  int32_t m;         /* rows per block at the top level; 0 = choose            */
                     /* (TPS_TRUNCATE: kept rows per window, even)             */
  int32_t m_reduced; /* rows per block at the recursive levels (>= 4); 0 =     */
                     /* choose (TPS_TRUNCATE: halo rows per side, even)        */
  int32_t streams;   /* S for tps_solve_host_async (1..32); 0 = choose         */
  int32_t max_iters; /* refinement iteration cap; 0 = 10                       */
  int64_t chunk;     /* rows per host-pipeline chunk; 0 = choose               */
  double tol;        /* refinement stop: ||delta||/||x|| <= tol; 0 = 1e-12     */
                     /* (TPS_TRUNCATE: the largest accepted error bound)       */
  uint32_t flags;    /* TPS_TUNE_* | TPS_TRACE | TPS_EXTERNAL_WORKSPACE |      */
                     /* TPS_GRAPH | TPS_ZERO_COPY | TPS_NO_ONCHIP |            */
                     /* TPS_TRUNCATE                                           */
  uint32_t reserved; /* must be 0                                              */
} tps_plan_desc;

typedef struct tps_plan_s* tps_plan_t;

typedef struct {
  int32_t status;        /* tps_status of the numeric checks since the last query */
  int32_t iterations;    /* refinement iterations of the last mixed solve         */
  int32_t m;             /* parameters the plan uses                              */
  int32_t m_reduced;
  int32_t streams;
  int32_t levels;        /* partition levels of the last solve launched level by  */
                         /* level (those before an on-chip solve)                 */
  int64_t chunk;
  double last_correction; /* ||delta||/||x|| of the last refinement step          */
  float stage_ms[4];     /* TPS_TRACE: stage 1, stage 2, stage 3, total (last solve) */
  size_t workspace_bytes;
  int32_t pageable_ok;   /* TPS_ZERO_COPY plans: 1 if pageable host memory is     */
                         /* accepted (the device reads it coherently), else 0     */
  int32_t onchip;        /* last solve: 0 all levels by separate launches; 1 the   */
                         /* whole system, 2 its reduced system, solved on chip     */
  int32_t refine_fused;  /* last mixed solve: 1 if its corrections ran fused into   */
                         /* level 0's Stage 1 / Stage 3 (residual formed in Stage 1, */
                         /* x += delta in Stage 3), 0 as separate passes            */
} tps_info;

/* Create a plan.  Validates `desc` (n_max >= 0, dtype, m 0 or >= 2, streams
 * 0 or 1..32, known flags, reserved == 0; TPS_ZERO_COPY needs host
 * residency, TPS_TRUNCATE device residency and a non-mixed dtype), resolves
 * zero parameters (predictor when TPS_TUNE_PREDICT is set, fixed defaults
 * otherwise), creates the streams and events of the host pipeline and,
 * unless TPS_EXTERNAL_WORKSPACE is set, allocates the device workspace.
 * Returns TPS_ERR_INVALID_ARG or TPS_ERR_UNSUPPORTED for a bad descriptor,
 * TPS_ERR_OOM if the workspace cannot be allocated.  On failure *out is
 * NULL. */
tps_status tps_plan(const tps_plan_desc* desc, tps_plan_t* out);

/* Release everything the plan owns (not a caller-supplied workspace).  The
 * caller must make sure no solve on the plan is still running. */
tps_status tps_plan_destroy(tps_plan_t plan);

/* Device workspace the plan needs for n_max / batch_max, in bytes. */
tps_status tps_workspace_size(tps_plan_t plan, size_t* bytes);

/* Hand the plan a caller-owned device buffer of at least
 * tps_workspace_size bytes (256-byte aligned).  Only for plans created with
 * TPS_EXTERNAL_WORKSPACE; the buffer must outlive every solve. */
tps_status tps_set_workspace(tps_plan_t plan, void* dev_ptr, size_t bytes);

/* Solve one system of n <= n_max rows held in device memory (Sec. 2.2,
 * Stages 1-3 on the GPU).  a, b, c, d, x: device pointers to n elements of
 * the plan's I/O type, 8-byte aligned for fp64, 4-byte for fp32.  Enqueues
 * the kernels on `stream` and returns; no host synchronisation, so it may
 * be captured into a CUDA graph (except TPS_MIXED_F32_F64, which reads its
 * convergence test back to the host after every correction).  With
 * TPS_GRAPH the plan captures the whole solve (every launch of Stages 1-3)
 * into a CUDA graph on a private stream at the first call with a given size,
 * geometry and set of pointers, and replays it as one graph launch while
 * they stay the same (also tps_solve_batched, whose offsets pointer is part
 * of the key); new pointers or sizes recapture.  With TPS_TRACE as well, or
 * in the host pipeline, only Stage 2 -- the recursive solve of the reduced
 * system, a chain of small launches that touches only the workspace -- is
 * captured, keyed by its level geometry, so the stage events stay apart.
 *
 * A system that fits in the GPU's shared memory (up to ~0.89 M rows in
 * fp64 and double-float, ~1.8 M in fp32 on 152 SMs; not for packed batches)
 * is solved by a single cooperative launch that reads a, b, c, d once and
 * writes x once: each CTA eliminates its rows on chip, one grid barrier,
 * every CTA solves the small system of CTA interface rows, and recovers its
 * rows on chip.  The reduced system of a larger solve takes the same path
 * once it fits.  TPS_NO_ONCHIP keeps every level on separate launches.
 * The grid barrier waits a bounded time: if the launch's CTAs cannot all
 * become resident (another such launch from another stream, or other
 * long-running work holding the SMs), the wait ends, the solve reports
 * TPS_ERR_TIMEOUT through tps_plan_query and the context stays usable; run
 * on-chip solves of different streams one after the other, or use
 * TPS_NO_ONCHIP for plans that run concurrently.
 *
 * TPS_MIXED_F32_F64: x0 from an fp32 elimination of the fp64 inputs, then
 * corrections until ||delta||/||x|| <= tol or max_iters.  Where the system
 * is solved level by level, each correction is one fused pass of the
 * partition method: Stage 1 forms r = d - A x in fp64 from the rows and the
 * current x (writing r to the workspace), Stage 3 adds the fp32 solution of
 * A delta = r to x in place (tps_info.refine_fused = 1); the single-launch
 * on-chip route keeps a separate residual pass, solve and update pass.
 *
 * TPS_TRUNCATE (device plans, fp64 / double-float / fp32; not the paper's
 * method, an approximation for strongly dominant systems): windows of m kept
 * rows are solved independently, each as the system on the window plus
 * m_reduced halo rows on either side with the couplings beyond cut; one
 * pass over the arrays, no reduced system across windows.  m (even) and
 * m_reduced (even) must satisfy m + 2 m_reduced <= 1792 (one CTA per
 * window, on chip) or m + 2 m_reduced = 32 mb with 8 <= mb <= 256 (one warp
 * per window: 32 blocks of mb rows, one per lane, the partition method
 * inside the warp, the blocks' row relations kept in a workspace buffer of
 * about 24 bytes per row, written once and read back once; at the default
 * window size about two thirds of it round-trip through DRAM); 0 chooses (the halo for
 * the plan's tol at a dominance factor max(|a|+|c|)/|b| of 3/4, one-warp
 * windows of 32 blocks of 256 rows).  Each window bounds its own error from
 * its dominance factor q and smallest |b|: (|a_cut| q^h + |c_cut| q^h) /
 * ((1 - q) min|b|) relative to max|x|; tps_plan_query reports the largest
 * bound of the last solve in last_correction and TPS_ERR_NO_CONVERGENCE if
 * it exceeds tol (default 1e-12).
 * The barrier waits a bounded time; if it runs out (which needs CTAs that
 * are not co-resident) the solve stops and tps_plan_query reports
 * TPS_ERR_TIMEOUT. */
tps_status tps_solve(tps_plan_t plan, int64_t n, const void* a, const void* b, const void* c,
                     const void* d, void* x, void* stream);

/* Solve `count` independent systems packed back to back: system s owns rows
 * offsets[s] .. offsets[s+1]-1.  offsets: device pointer to count+1 int64
 * values, offsets[0] = 0, non-decreasing, offsets[count] <= n_max;
 * host_offsets: the same values in host memory (used to build the work
 * list; may be NULL, then the offsets are read back with a synchronous
 * copy).  count <= batch_max. */
tps_status tps_solve_batched(tps_plan_t plan, int64_t count, const int64_t* offsets,
                             const int64_t* host_offsets, const void* a, const void* b,
                             const void* c, const void* d, void* x, void* stream);

/* Solve one system held in pinned host memory (cudaHostAlloc /
 * cudaHostRegister): copies the rows to the device in chunks on the plan's
 * S streams, overlapping each chunk's host-to-device copy with the Stage-1
 * kernel of the previous chunk; then Stage 2; then per chunk Stage 3 and the
 * device-to-host copy of x (Sec. 2.2, Eq. 2).  The device keeps its copy of
 * a, b, c, d between the stages, so nothing is uploaded twice.  Work is
 * ordered after everything already in `stream`, and `stream` waits for all
 * of it; the call returns after enqueueing.  Pageable memory gives
 * TPS_ERR_INVALID_ARG.
 *
 * With TPS_ZERO_COPY no copy engine is used: the same chunked pipeline moves
 * each chunk with a streaming kernel whose threads load from and store to
 * host memory directly (consecutive threads, consecutive 16-byte vectors),
 * concurrent with the stage kernels of other chunks.  The link carries the
 * same bytes (each input once up, x once down).  Host arrays may then be
 * pinned memory, or ordinary pageable memory where the device has coherent
 * access to it (cudaDevAttrPageableMemoryAccess, e.g. Grace-based systems;
 * tps_plan_query reports it); elsewhere pageable memory gives
 * TPS_ERR_INVALID_ARG.  The pages must stay mapped until `stream`
 * completes.  mixed dtype: TPS_ERR_UNSUPPORTED. */
tps_status tps_solve_host_async(tps_plan_t plan, int64_t n, const void* a, const void* b,
                                const void* c, const void* d, void* x, void* stream);

/* Solve `count` independent host-resident systems of n rows each, in order,
 * overlapping consecutive systems: each system runs the pipeline of
 * tps_solve_host_async, and consecutive systems alternate between two sets
 * of device buffers, workspaces and S streams (the plan's own and those of
 * a twin plan that tps_plan makes for TPS_HOST_OVERLAP), so system k+1
 * uploads while system k finishes Stage 3 and downloads: the link carries
 * both directions at once.  One system alone cannot do this, since none of
 * its x can leave before all of its rows have arrived (Stage 2 couples
 * them).
 *   plan        made with residency TPS_HOST_PINNED and TPS_HOST_OVERLAP
 *               (which implies TPS_NO_ONCHIP: two on-chip cooperative launches
 *               of different systems may not run at once; not with
 *               TPS_EXTERNAL_WORKSPACE); the twin follows the plan's m,
 *               m_reduced, S and chunk, including tps_autotune's choice
 *   n           rows of every system, 0 .. n_max
 *   a, b, c, d  count host pointers each (inputs, as for
 *               tps_solve_host_async); systems may share inputs
 *   x           count host pointers (outputs); x[k] must not overlap x[k+1]
 *               or any input of systems k-1, k, k+1 (TPS_ERR_INVALID_ARG)
 * Stream-ordered on `stream` as one operation (it starts after the work
 * already in `stream`, and `stream` waits for every system); returns after
 * enqueueing.  If the arrays of system k are rejected (the checks of
 * tps_solve_host_async), systems 0 .. k-1 stay enqueued and `stream` still
 * waits for them.  Numeric status of all systems: tps_plan_query on the
 * plan. */
tps_status tps_solve_host_many_async(tps_plan_t plan, int64_t count, int64_t n,
                                     const void* const* a, const void* const* b,
                                     const void* const* c, const void* const* d,
                                     void* const* x, void* stream);

/* Largest system tps_solve_noalloc accepts, in rows. */
#define TPS_NOALLOC_MAX_ROWS 262144

/* The device-resident solve of tps_solve for callers that cannot allocate
 * device memory: code inside a framework whose caching allocator must own
 * every device buffer, code running under a fixed device-memory budget, or
 * a latency-critical loop where a cudaMalloc (which may synchronise the
 * device) is not acceptable.  It needs no plan and
 * allocates nothing: its scratch (reduced systems, Stage-1 checkpoints, a
 * status word) is one fixed 2 MiB array in device memory that every GPU
 * loading libtps holds until the process exits.  The paper has no
 * counterpart to this entry point.
 *   dtype       TPS_F64, TPS_F64_DF or TPS_F32 (as in tps_plan_desc)
 *   n           0 .. TPS_NOALLOC_MAX_ROWS; larger n gives TPS_ERR_INVALID_ARG
 *   a, b, c, d  device inputs, x device output (n elements of the I/O type;
 *               x must not overlap an input), owned by the caller, on the
 *               current device; only alignment and overlap are checked (no
 *               pointer queries on this path)
 *   status_out  optional device int32 that receives TPS_OK,
 *               TPS_ERR_ZERO_PIVOT, TPS_ERR_TIMEOUT or TPS_ERR_RANGE when
 *               the solve has run (NULL: not reported)
 *   stream      cudaStream_t as void*
 * A system that fits in shared memory (every accepted size on a 152-SM
 * GB300) is solved by the single-launch on-chip solve (see tps_solve);
 * otherwise fixed parameters m = 64 at the top level, 32 below.  The first
 * call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current.  Every call overwrites
 * the shared scratch, so calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller. */
tps_status tps_solve_noalloc(int32_t dtype, int64_t n, const void* a, const void* b,
                             const void* c, const void* d, void* x, int32_t* status_out,
                             void* stream);

/* ---------------------------------------------------------------------------
 * Launch-parameter selection.  The paper fits a model of the optimum stream
 * count (Sec. 2.4: Eq. 4 and Eq. 7 fed into Eq. 6); this library adds a small
 * learned predictor, an MLP trained on the GPU on timings the solver itself
 * produced, that chooses the block size m, the stream count S and the chunk
 * size from (log2 n, log2 batch, dtype, residency).
 * ------------------------------------------------------------------------- */
#define TPS_MLP_IN 4
#define TPS_MLP_HIDDEN 64
#define TPS_MLP_OUT 3
/* [W1 (64x4), b1 (64), W2 (64x64), b2 (64), W3 (3x64), b3 (3)], row-major
 * [out][in], fp32 */
#define TPS_MLP_NPARAMS 4675

/* fp32 scratch (in floats) that tps_mlp_forward / tps_mlp_loss_backward need
 * for a batch of `batch` samples. */
size_t tps_mlp_workspace_floats(int32_t batch);

/* Y[batch][3] = MLP(X[batch][4]) on the device (two ReLU hidden layers of
 * 64).  All pointers are device memory owned by the caller; `work` holds
 * tps_mlp_workspace_floats(batch) floats. */
tps_status tps_mlp_forward(const float* params, int32_t batch, const float* X, float* Y,
                           float* work, void* stream);

/* Forward pass, loss L = mean((Y - T)^2) over batch and outputs (written to
 * *loss, device, may be NULL) and the gradient dL/dparams (grads, device,
 * TPS_MLP_NPARAMS floats, overwritten). */
tps_status tps_mlp_loss_backward(const float* params, int32_t batch, const float* X,
                                 const float* T, float* grads, float* loss, float* work,
                                 void* stream);

/* One Adam step (Kingma and Ba) on the device: m, v are the moment buffers
 * (TPS_MLP_NPARAMS floats, zero before step t = 1). */
tps_status tps_mlp_adam_step(float* params, const float* grads, float* m, float* v, int32_t t,
                             float lr, float beta1, float beta2, float eps, void* stream);

/* The same forward pass on the host for one sample (x[4] -> y[3]); the
 * multiply-add order matches the device kernels, so results agree bit for
 * bit. */
void tps_mlp_forward_host(const float* params, const float* x, float* y);

/* Fill m, streams and chunk for `desc` from the installed predictor weights
 * ($TPS_PREDICTOR_WEIGHTS, else predictor/weights.bin beside libtps.so).
 * Returns 0 on success, 1 when no weights are installed, 2 on bad
 * arguments.  chunk = 0 means one chunk per stream. */
int tps_predict_params(const tps_plan_desc* desc, int32_t* m, int32_t* streams,
                       int64_t* chunk);

/* 1 if predictor weights could be loaded, else 0. */
int tps_predict_available(void);

/* Load predictor weights from `path` (the training driver's file format),
 * replacing any loaded ones.  Returns 0 on success, 1 if the file is
 * missing or malformed, 2 for a NULL path. */
int tps_predict_load(const char* path);

/* Exhaustive search: time tps_solve (count == 0: one system of n rows) or
 * tps_solve_batched (count > 0, offsets as there) on the caller's data for
 * every block size m in {16, 32, ..., 1024} whose workspace fits the plan,
 * `reps` timed solves each after one warm-up, and keep the fastest m in the
 * plan.  A plan created with TPS_TUNE_EXHAUSTIVE sizes its workspace for the
 * whole grid.  Synchronises `stream`; x is overwritten.  *best_m and
 * *best_ms (may be NULL) receive the choice and its mean time.
 * For a host-residency plan (count must be 0, a..x pinned or, with
 * TPS_ZERO_COPY, host memory as tps_solve_host_async accepts) the search is
 * over the stream count S in {1, 2, 4, 8, 16, 32} and the chunk in
 * {n/S, 2^22, 2^24 rows} through tps_solve_host_async instead, and the
 * fastest (S, chunk) is kept (tps_plan_query reports them); the plan's
 * stream set grows to 32 streams. */
tps_status tps_autotune(tps_plan_t plan, int64_t n, int64_t count, const int64_t* offsets,
                        const int64_t* host_offsets, const void* a, const void* b,
                        const void* c, const void* d, void* x, void* stream, int32_t reps,
                        int32_t* best_m, float* best_ms);

/* The paper's optimum-stream rule (Sec. 2.4, Eq. 6) with the sum model of
 * Eq. 4 (sum_model[2]: slope, intercept) and the overhead models of Eq. 7
 * (small[3]: size, log10 S and constant coefficients, for size <= split;
 * big[3]: size and constant inside the log2(S^(4/3)) factor, then the
 * constant, for size > split).  NULL coefficient pointers select the
 * paper's RTX 2080 Ti values; split <= 0 selects 1e6.  Returns S in
 * {1, 2, 4, 8, 16, 32}: among S with T_overhead(S) < (S-1)/S * sum the one
 * with the largest slack, or 1 when none qualifies. */
int32_t tps_paper_predict_streams(double size, const double* sum_model, const double* small,
                                  const double* big, double split);

/* Report the plan's parameters and the numeric status of the solves since
 * the previous query (synchronises the plan's last stream, reads the device
 * status word and clears it).  Several conditions at once report the first
 * of TPS_ERR_ZERO_PIVOT, TPS_ERR_TIMEOUT, TPS_ERR_RANGE,
 * TPS_ERR_NO_CONVERGENCE.  Every dtype reports TPS_ERR_RANGE for an x that
 * is not finite. */
tps_status tps_plan_query(tps_plan_t plan, tps_info* out);

/* Measurement aid (the paper has no counterpart): the current device's
 * fp64 instruction rates -- fused multiply-add, multiply and add, in
 * thread instructions per second (any pointer may be NULL) -- from
 * synthetic kernels of independent dependency chains on every SM (for each
 * kind the best of ten launches of a few ms at two occupancies, on the
 * legacy default stream; allocates and frees a small buffer and
 * synchronises the device).  They are the peaks against which the plain
 * fp64 solve, bound by the fp64 pipe on GB300, is reported. */
tps_status tps_measure_fp64_rates(double* fma_per_s, double* mul_per_s, double* add_per_s);

/* Static description of a status code. */
const char* tps_status_string(tps_status s);

/* Library version: major * 10000 + minor * 100 + patch. */
int tps_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TPS_H */
