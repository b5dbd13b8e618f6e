/*
 * CPU oracle for the tridiagonal partition method -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs may load or call this library.  The product path (the CUDA
 * library and its Python binding) never does, and shares no code with it.
 *
 * Everything is plain, serial, IEEE fp64 C, compiled with -ffp-contract=off
 * so no multiply-add is ever fused.  The system is
 *
 *     a[i]*x[i-1] + b[i]*x[i] + c[i]*x[i+1] = d[i],   i = 0 .. n-1,
 *
 * with a[0] and c[n-1] never read.
 *
 * What the paper fixes and what is a reading:
 *   - Sec. 1: the partition method (Austin et al. 2004) splits the
 *     tridiagonal matrix into sub-matrices whose smaller systems are solved
 *     in parallel.  The paper prints no formulas for it.
 *   - Sec. 2.2: the method has three stages -- Stage 1 and Stage 3 per
 *     sub-system, Stage 2 a reduced (interface) system in between.
 *   - Sec. 2.2 / Table 1: after Stage 1 four reduced-coefficient arrays go
 *     down to the host and one reduced-solution array comes back
 *     (T1^D2H / T3^H2D is about 4 at every size), which is what two
 *     interface unknowns per block with a tridiagonal reduced system give.
 *   The partition solver below takes that reading: blocks of m consecutive
 *   rows, the first and last row of each block are its interface unknowns,
 *   the interior rows are eliminated (Stage 1), the reduced tridiagonal
 *   system in the interface unknowns is solved (Stage 2, here by Thomas),
 *   and the interior is recovered (Stage 3).  Being a direct method it
 *   returns A^{-1} d up to rounding, which is how the tests pin it.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ZERO_PIVOT 1
#define ORC_BAD_ARG 2
#define ORC_NO_MEMORY 3

/* ------------------------------------------------------------------------
 * Thomas algorithm (textbook Gaussian elimination without pivoting for a
 * tridiagonal matrix).  Stable for strictly diagonally dominant A.
 *   forward:  beta_0 = b_0,  y_0 = d_0 / beta_0
 *             gamma_{i-1} = c_{i-1} / beta_{i-1}
 *             beta_i = b_i - a_i * gamma_{i-1}
 *             y_i    = (d_i - a_i * y_{i-1}) / beta_i
 *   backward: x_{n-1} = y_{n-1},  x_i = y_i - gamma_i * x_{i+1}
 * gamma is kept in the caller-provided scratch (n doubles) or malloc'ed.
 * ---------------------------------------------------------------------- */
static int thomas_core(int64_t n, const double *a, const double *b, const double *c,
                       const double *d, double *x, double *gamma) {
  if (n <= 0) return ORC_OK;
  double beta = b[0];
  if (beta == 0.0 || !isfinite(beta)) return ORC_ZERO_PIVOT;
  x[0] = d[0] / beta;
  for (int64_t i = 1; i < n; ++i) {
    gamma[i - 1] = c[i - 1] / beta;
    beta = b[i] - a[i] * gamma[i - 1];
    if (beta == 0.0 || !isfinite(beta)) return ORC_ZERO_PIVOT;
    x[i] = (d[i] - a[i] * x[i - 1]) / beta;
  }
  for (int64_t i = n - 2; i >= 0; --i) x[i] = x[i] - gamma[i] * x[i + 1];
  return ORC_OK;
}

int orc_thomas(int64_t n, const double *a, const double *b, const double *c, const double *d,
               double *x) {
  if (n < 0) return ORC_BAD_ARG;
  if (n == 0) return ORC_OK;
  double *gamma = (double *)malloc((size_t)n * sizeof(double));
  if (!gamma) return ORC_NO_MEMORY;
  int st = thomas_core(n, a, b, c, d, x, gamma);
  free(gamma);
  return st;
}

/* Independent systems packed back to back: system s owns rows
 * offsets[s] .. offsets[s+1]-1; a at each system's first row and c at its
 * last row are never read, so the systems never couple. */
int orc_thomas_batched(int64_t count, const int64_t *offsets, const double *a, const double *b,
                       const double *c, const double *d, double *x) {
  if (count < 0) return ORC_BAD_ARG;
  int64_t nmax = 0;
  for (int64_t s = 0; s < count; ++s) {
    int64_t len = offsets[s + 1] - offsets[s];
    if (len < 0) return ORC_BAD_ARG;
    if (len > nmax) nmax = len;
  }
  double *gamma = (double *)malloc((size_t)(nmax > 0 ? nmax : 1) * sizeof(double));
  if (!gamma) return ORC_NO_MEMORY;
  int st = ORC_OK;
  for (int64_t s = 0; s < count && st == ORC_OK; ++s) {
    int64_t o = offsets[s], len = offsets[s + 1] - offsets[s];
    st = thomas_core(len, a + o, b + o, c + o, d + o, x + o, gamma);
  }
  free(gamma);
  return st;
}

/* ------------------------------------------------------------------------
 * Partition method, serial, step by step (reading of Sec. 1 / Sec. 2.2).
 *
 * Blocks k = 0 .. p-1 cover rows r0 = k*m .. r1 = min(r0+m, n) - 1, with
 * length L = r1 - r0 + 1 (only the last block can be shorter than m).
 * Interface unknowns: f_k = x[r0] and l_k = x[r1] (one unknown if L = 1).
 *
 * Stage 1, for L >= 3: the interior rows r0+1 .. r1-1 form a tridiagonal
 * matrix T.  Moving the interface terms to the right-hand side gives
 *     x_int = y - v * f_k - w * l_k,
 *     T y = d_int,  T v = a[r0+1] e_1,  T w = c[r1-1] e_last,
 * solved here by Thomas with three right-hand sides.  Substituting the
 * first and last interior rows into the block's rows r0 and r1 gives its
 * two reduced equations
 *     a[r0] l_{k-1} + (b[r0] - c[r0] v_1) f_k - c[r0] w_1 l_k = d[r0] - c[r0] y_1
 *     -a[r1] v_e f_k + (b[r1] - a[r1] w_e) l_k + c[r1] f_{k+1} = d[r1] - a[r1] y_e
 * For L = 2 the two reduced equations are the block's own two rows, and
 * for L = 1 its single row.
 *
 * Stage 2: the reduced unknowns in the order f_0, l_0, f_1, l_1, ... form a
 * tridiagonal system (a Schur complement of A, hence again strictly
 * diagonally dominant when A is); it is solved by Thomas.
 *
 * Stage 3: x_int = y - v f_k - w l_k for every block.
 *
 * The reduced system can be returned through red_* (each of length
 * orc_partition_reduced_size(n, m)) when those pointers are non-NULL.
 * ---------------------------------------------------------------------- */
int64_t orc_partition_reduced_size(int64_t n, int64_t m) {
  if (n <= 0 || m < 2) return 0;
  int64_t p = (n + m - 1) / m;
  int64_t last = n - (p - 1) * m;
  return 2 * p - (last == 1 ? 1 : 0);
}

/* Stage 1 of block k (rows r0 .. r1, L = r1 - r0 + 1): y, v, w of its
 * interior rows and its reduced rows 2k, 2k+1.  gam: m doubles of scratch.
 * Blocks touch disjoint parts of y, v, w and the reduced arrays. */
static int stage1_block(int64_t k, int64_t p, int64_t n, int64_t m, const double *a,
                        const double *b, const double *c, const double *d, double *y,
                        double *v, double *w, double *ra, double *rb, double *rc, double *rd,
                        double *gam) {
  const int64_t r0 = k * m;
  const int64_t r1 = (r0 + m < n ? r0 + m : n) - 1;
  const int64_t L = r1 - r0 + 1;
  const int64_t jf = 2 * k;      /* reduced index of f_k */
  const int64_t jl = 2 * k + 1;  /* reduced index of l_k (if L >= 2) */
  if (L >= 3) {
    /* Thomas on T with the three right-hand sides d_int, a[r0+1] e_1,
     * c[r1-1] e_last, column by column, sharing the pivots. */
    const int64_t i0 = r0 + 1, ie = r1 - 1, ni = ie - i0 + 1;
    double beta = b[i0];
    if (beta == 0.0 || !isfinite(beta)) return ORC_ZERO_PIVOT;
    y[i0] = d[i0] / beta;
    v[i0] = a[i0] / beta;
    w[i0] = (ni == 1 ? c[ie] : 0.0) / beta;
    for (int64_t t = 1; t < ni; ++t) {
      const int64_t i = i0 + t;
      gam[t - 1] = c[i - 1] / beta;
      beta = b[i] - a[i] * gam[t - 1];
      if (beta == 0.0 || !isfinite(beta)) return ORC_ZERO_PIVOT;
      const double rhs_w = (i == ie) ? c[ie] : 0.0;
      y[i] = (d[i] - a[i] * y[i - 1]) / beta;
      v[i] = (0.0 - a[i] * v[i - 1]) / beta;
      w[i] = (rhs_w - a[i] * w[i - 1]) / beta;
    }
    for (int64_t t = ni - 2; t >= 0; --t) {
      const int64_t i = i0 + t;
      y[i] = y[i] - gam[t] * y[i + 1];
      v[i] = v[i] - gam[t] * v[i + 1];
      w[i] = w[i] - gam[t] * w[i + 1];
    }
    /* first reduced row (unknowns l_{k-1}, f_k, l_k) */
    ra[jf] = (k > 0) ? a[r0] : 0.0;
    rb[jf] = b[r0] - c[r0] * v[i0];
    rc[jf] = 0.0 - c[r0] * w[i0];
    rd[jf] = d[r0] - c[r0] * y[i0];
    /* last reduced row (unknowns f_k, l_k, f_{k+1}) */
    ra[jl] = 0.0 - a[r1] * v[ie];
    rb[jl] = b[r1] - a[r1] * w[ie];
    rc[jl] = (k < p - 1) ? c[r1] : 0.0;
    rd[jl] = d[r1] - a[r1] * y[ie];
  } else if (L == 2) {
    ra[jf] = (k > 0) ? a[r0] : 0.0;
    rb[jf] = b[r0];
    rc[jf] = c[r0];
    rd[jf] = d[r0];
    ra[jl] = a[r1];
    rb[jl] = b[r1];
    rc[jl] = (k < p - 1) ? c[r1] : 0.0;
    rd[jl] = d[r1];
  } else { /* L == 1: only the last block can be this short */
    ra[jf] = (k > 0) ? a[r0] : 0.0;
    rb[jf] = b[r0];
    rc[jf] = 0.0;
    rd[jf] = d[r0];
  }
  return ORC_OK;
}

/* Stage 3 of block k: x_int = y - v f_k - w l_k from the reduced solution. */
static void stage3_block(int64_t k, int64_t n, int64_t m, const double *y, const double *v,
                         const double *w, const double *rx, double *x) {
  const int64_t r0 = k * m;
  const int64_t r1 = (r0 + m < n ? r0 + m : n) - 1;
  const int64_t L = r1 - r0 + 1;
  const double f = rx[2 * k];
  const double l = (L >= 2) ? rx[2 * k + 1] : f;
  x[r0] = f;
  x[r1] = l;
  for (int64_t i = r0 + 1; i <= r1 - 1; ++i) x[i] = y[i] - v[i] * f - w[i] * l;
}

/* The work arrays of one partition solve. */
typedef struct {
  int64_t n, m, p, nr;
  const double *a, *b, *c, *d;
  double *x, *y, *v, *w, *ra, *rb, *rc, *rd, *rx;
} part_ctx;

static int part_alloc(part_ctx *P, int64_t n, int64_t m, const double *a, const double *b,
                      const double *c, const double *d, double *x) {
  memset(P, 0, sizeof(*P));
  P->n = n; P->m = m; P->p = (n + m - 1) / m;
  P->nr = orc_partition_reduced_size(n, m);
  P->a = a; P->b = b; P->c = c; P->d = d; P->x = x;
  P->y = (double *)calloc((size_t)n, sizeof(double));
  P->v = (double *)calloc((size_t)n, sizeof(double));
  P->w = (double *)calloc((size_t)n, sizeof(double));
  P->ra = (double *)calloc((size_t)P->nr, sizeof(double));
  P->rb = (double *)calloc((size_t)P->nr, sizeof(double));
  P->rc = (double *)calloc((size_t)P->nr, sizeof(double));
  P->rd = (double *)calloc((size_t)P->nr, sizeof(double));
  P->rx = (double *)calloc((size_t)P->nr, sizeof(double));
  return (P->y && P->v && P->w && P->ra && P->rb && P->rc && P->rd && P->rx) ? ORC_OK
                                                                              : ORC_NO_MEMORY;
}

static void part_free(part_ctx *P) {
  free(P->y); free(P->v); free(P->w);
  free(P->ra); free(P->rb); free(P->rc); free(P->rd); free(P->rx);
}

int orc_partition_ex(int64_t n, int64_t m, const double *a, const double *b, const double *c,
                     const double *d, double *x, double *red_a, double *red_b, double *red_c,
                     double *red_d) {
  if (n < 0 || m < 2) return ORC_BAD_ARG;
  if (n == 0) return ORC_OK;
  part_ctx P;
  int st = part_alloc(&P, n, m, a, b, c, d, x);
  double *gam = (double *)malloc((size_t)m * sizeof(double));
  if (st != ORC_OK || !gam) {
    st = ORC_NO_MEMORY;
    goto done;
  }
  /* ---- Stage 1 ---- */
  for (int64_t k = 0; k < P.p && st == ORC_OK; ++k)
    st = stage1_block(k, P.p, n, m, a, b, c, d, P.y, P.v, P.w, P.ra, P.rb, P.rc, P.rd, gam);
  if (st != ORC_OK) goto done;
  /* ---- Stage 2: reduced system by Thomas ---- */
  st = orc_thomas(P.nr, P.ra, P.rb, P.rc, P.rd, P.rx);
  if (st != ORC_OK) goto done;
  /* ---- Stage 3 ---- */
  for (int64_t k = 0; k < P.p; ++k) stage3_block(k, n, m, P.y, P.v, P.w, P.rx, x);
  if (red_a) memcpy(red_a, P.ra, (size_t)P.nr * sizeof(double));
  if (red_b) memcpy(red_b, P.rb, (size_t)P.nr * sizeof(double));
  if (red_c) memcpy(red_c, P.rc, (size_t)P.nr * sizeof(double));
  if (red_d) memcpy(red_d, P.rd, (size_t)P.nr * sizeof(double));
done:
  part_free(&P);
  free(gam);
  return st;
}

/* ------------------------------------------------------------------------
 * The same partition solve with Stages 1 and 3 spread over `threads` host
 * threads (each a contiguous run of blocks; Stage 2 stays serial): the
 * multi-core CPU baseline.  Per block the arithmetic is that of
 * orc_partition_ex, in the same order, so the result is bit-identical.
 * ---------------------------------------------------------------------- */
typedef struct {
  part_ctx *P;
  int64_t k0, k1;
  int stage, status;
} part_job;

static void *part_worker(void *arg) {
  part_job *J = (part_job *)arg;
  part_ctx *P = J->P;
  J->status = ORC_OK;
  if (J->stage == 1) {
    double *gam = (double *)malloc((size_t)P->m * sizeof(double));
    if (!gam) { J->status = ORC_NO_MEMORY; return NULL; }
    for (int64_t k = J->k0; k < J->k1 && J->status == ORC_OK; ++k)
      J->status = stage1_block(k, P->p, P->n, P->m, P->a, P->b, P->c, P->d, P->y, P->v, P->w,
                               P->ra, P->rb, P->rc, P->rd, gam);
    free(gam);
  } else {
    for (int64_t k = J->k0; k < J->k1; ++k)
      stage3_block(k, P->n, P->m, P->y, P->v, P->w, P->rx, P->x);
  }
  return NULL;
}

static int part_parallel(part_ctx *P, int stage, int threads) {
  pthread_t tid[256];
  part_job job[256];
  if (threads > 256) threads = 256;
  if (threads < 1) threads = 1;
  int started = 0, st = ORC_OK;
  for (int t = 0; t < threads; ++t) {
    job[t].P = P;
    job[t].stage = stage;
    job[t].k0 = P->p * t / threads;
    job[t].k1 = P->p * (t + 1) / threads;
    job[t].status = ORC_OK;
    if (pthread_create(&tid[t], NULL, part_worker, &job[t]) != 0) {
      part_worker(&job[t]);  /* run it on this thread instead */
      if (job[t].status != ORC_OK) st = job[t].status;
      tid[t] = 0;
      continue;
    }
    ++started;
  }
  for (int t = 0; t < threads; ++t) {
    if (tid[t]) {
      pthread_join(tid[t], NULL);
      if (job[t].status != ORC_OK) st = job[t].status;
    }
  }
  (void)started;
  return st;
}

int orc_partition_threaded(int64_t n, int64_t m, const double *a, const double *b,
                           const double *c, const double *d, double *x, int threads) {
  if (n < 0 || m < 2 || threads < 1) return ORC_BAD_ARG;
  if (n == 0) return ORC_OK;
  part_ctx P;
  int st = part_alloc(&P, n, m, a, b, c, d, x);
  if (st == ORC_OK) st = part_parallel(&P, 1, threads);
  if (st == ORC_OK) st = orc_thomas(P.nr, P.ra, P.rb, P.rc, P.rd, P.rx);
  if (st == ORC_OK) st = part_parallel(&P, 3, threads);
  part_free(&P);
  return st;
}

int orc_partition(int64_t n, int64_t m, const double *a, const double *b, const double *c,
                  const double *d, double *x) {
  return orc_partition_ex(n, m, a, b, c, d, x, NULL, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------------
 * Dense Gaussian elimination with partial pivoting (row interchanges), the
 * textbook LU route, for small n.  The tridiagonal matrix is expanded into
 * an n x n row-major array first; n is limited to 512 to keep it small.
 * ---------------------------------------------------------------------- */
int orc_dense_ge(int64_t n, const double *a, const double *b, const double *c, const double *d,
                 double *x) {
  if (n < 0 || n > 512) return ORC_BAD_ARG;
  if (n == 0) return ORC_OK;
  double *M = (double *)calloc((size_t)(n * n), sizeof(double));
  double *r = (double *)malloc((size_t)n * sizeof(double));
  if (!M || !r) { free(M); free(r); return ORC_NO_MEMORY; }
  for (int64_t i = 0; i < n; ++i) {
    if (i > 0) M[i * n + i - 1] = a[i];
    M[i * n + i] = b[i];
    if (i < n - 1) M[i * n + i + 1] = c[i];
    r[i] = d[i];
  }
  int st = ORC_OK;
  for (int64_t k = 0; k < n; ++k) {
    int64_t piv = k;
    double best = fabs(M[k * n + k]);
    for (int64_t i = k + 1; i < n; ++i)
      if (fabs(M[i * n + k]) > best) { best = fabs(M[i * n + k]); piv = i; }
    if (best == 0.0) { st = ORC_ZERO_PIVOT; break; }
    if (piv != k) {
      for (int64_t j = 0; j < n; ++j) {
        double t = M[k * n + j]; M[k * n + j] = M[piv * n + j]; M[piv * n + j] = t;
      }
      double t = r[k]; r[k] = r[piv]; r[piv] = t;
    }
    for (int64_t i = k + 1; i < n; ++i) {
      double lik = M[i * n + k] / M[k * n + k];
      if (lik == 0.0) continue;
      for (int64_t j = k; j < n; ++j) M[i * n + j] -= lik * M[k * n + j];
      r[i] -= lik * r[k];
    }
  }
  if (st == ORC_OK) {
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = r[i];
      for (int64_t j = i + 1; j < n; ++j) s -= M[i * n + j] * x[j];
      x[i] = s / M[i * n + i];
    }
  }
  free(M); free(r);
  return st;
}

/* r = d - A x in fp64, products summed left to right. */
void orc_residual(int64_t n, const double *a, const double *b, const double *c, const double *d,
                  const double *x, double *r) {
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i] * x[i];
    if (i > 0) s = s + a[i] * x[i - 1];
    if (i < n - 1) s = s + c[i] * x[i + 1];
    r[i] = d[i] - s;
  }
}

/* max_i |u_i - v_i| and max_i |v_i| (the infinity norms used for the
 * relative forward error ||u - v|| / ||v||). */
void orc_maxabs_diff(int64_t n, const double *u, const double *v, double *out_diff,
                     double *out_ref) {
  double md = 0.0, mr = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double dd = fabs(u[i] - v[i]);
    double rr = fabs(v[i]);
    if (dd > md || dd != dd) md = (dd != dd) ? INFINITY : dd;
    if (rr > mr) mr = rr;
  }
  *out_diff = md;
  *out_ref = mr;
}

/* ------------------------------------------------------------------------
 * Thomas in IEEE binary32 arithmetic (same recurrences as thomas_core).
 * Used by the step-by-step mixed-precision refinement oracle, where the
 * inner solve of the correction equation is done in single precision.
 * ---------------------------------------------------------------------- */
int orc_thomas_f32(int64_t n, const float *a, const float *b, const float *c, const float *d,
                   float *x) {
  if (n < 0) return ORC_BAD_ARG;
  if (n == 0) return ORC_OK;
  float *gamma = (float *)malloc((size_t)n * sizeof(float));
  if (!gamma) return ORC_NO_MEMORY;
  int st = ORC_OK;
  float beta = b[0];
  if (beta == 0.0f || !isfinite(beta)) st = ORC_ZERO_PIVOT;
  if (st == ORC_OK) {
    x[0] = d[0] / beta;
    for (int64_t i = 1; i < n; ++i) {
      gamma[i - 1] = c[i - 1] / beta;
      beta = b[i] - a[i] * gamma[i - 1];
      if (beta == 0.0f || !isfinite(beta)) { st = ORC_ZERO_PIVOT; break; }
      x[i] = (d[i] - a[i] * x[i - 1]) / beta;
    }
  }
  if (st == ORC_OK)
    for (int64_t i = n - 2; i >= 0; --i) x[i] = x[i] - gamma[i] * x[i + 1];
  free(gamma);
  return st;
}
