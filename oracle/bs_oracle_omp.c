/*
 * bs_oracle_omp.c -- the oracle's plain BS1-BS7 loops spread over the host
 * cores with OpenMP, for the benchmark's multi-core CPU baseline.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of this directory: the benchmark's
 * CPU-baseline leg and the tests are the only callers; the GPU library never
 * links or loads it.
 *
 * Each loop is the oracle's definition (Table 1, eq. scatter_def) with its
 * index range split statically over the threads:
 *  - BS1, BS2, BS7 and the update of BS5: the same per-entry arithmetic as
 *    bs_oracle.c, so the results are bitwise the single-threaded ones;
 *  - BS3, BS4 and the r.r of BS5: every thread runs the doubled-precision
 *    Dot2 of Ogita, Rump & Oishi (2005) over its contiguous chunk, and the
 *    chunk results are combined in thread order, again as a Dot2-style
 *    compensated sum -- as accurate as the single-threaded Dot2, not bitwise
 *    the same;
 *  - BS6: every global node sums its local copies in ascending local index
 *    from +0.0 (the oracle's order), rows split over the threads; the copies
 *    of each row come from the CSR of Z^T (rowStarts, colIds ascending),
 *    built once before timing (bso_csr in bs_oracle.c), so the sums are
 *    bitwise the single-threaded ones.
 * Compiled with -fopenmp -O2 -ffp-contract=off.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>

static void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double z = x - a;
  *s = x;
  *e = (a - (x - z)) + (b - z);
}

static void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *p = x;
  *e = fma(a, b, -x);
}

/* Dot2 over [lo, hi): the compensated pair (p, s). */
static void dot2_chunk(int64_t lo, int64_t hi, const double *x, const double *y, double *P,
                       double *S) {
  double p = 0.0, s = 0.0, h, r, q;
  for (int64_t i = lo; i < hi; ++i) {
    two_prod(x[i], y[i], &h, &r);
    two_sum(p, h, &p, &q);
    s = s + (q + r);
  }
  *P = p;
  *S = s;
}

#define MAXT 1024

/* Dot2 with the index range split over the threads; chunk pairs combined in
 * thread order with TwoSum on the leading parts. */
static double dot2_omp(int64_t n, const double *x, const double *y) {
  double P[MAXT], S[MAXT];
  int nt = 1;
#pragma omp parallel
  {
#pragma omp single
    nt = omp_get_num_threads() < MAXT ? omp_get_num_threads() : MAXT;
    const int t = omp_get_thread_num();
    if (t < nt) {
      const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
      dot2_chunk(lo, hi, x, y, &P[t], &S[t]);
    }
  }
  double p = 0.0, s = 0.0, q;
  for (int t = 0; t < nt; ++t) {
    two_sum(p, P[t], &p, &q);
    s = s + (q + S[t]);
  }
  return p + s;
}

int bso_omp_threads(void) { return omp_get_max_threads(); }

void bso_omp_copy(int64_t n, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) y[i] = x[i];
}

void bso_omp_axpy(int64_t n, double alpha, const double *x, double beta, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) y[i] = fma(alpha, x[i], beta * y[i]);
}

void bso_omp_norm(int64_t n, const double *x, double *out) {
  const double s = dot2_omp(n, x, x);
  out[0] = s;
  out[1] = sqrt(s);
}

double bso_omp_dot(int64_t n, const double *x, const double *y) { return dot2_omp(n, x, y); }

double bso_omp_cg_update(int64_t n, double alpha, const double *p, const double *Ap, double *x,
                         double *r) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, Ap[i], r[i]);
  }
  return dot2_omp(n, r, r);
}

void bso_omp_scatter(int64_t NL, const int32_t *ids, const double *qG, double *qL) {
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < NL; ++l)
    if (ids[l] >= 0) qL[l] = qG[ids[l]];
}

void bso_omp_gather_csr(int64_t NG, const int32_t *row_starts, const int32_t *col_ids,
                        const double *qL, double *qG) {
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < NG; ++g) {
    double s = 0.0;
    for (int32_t k = row_starts[g]; k < row_starts[g + 1]; ++k) s = s + qL[col_ids[k]];
    qG[g] = s;
  }
}
