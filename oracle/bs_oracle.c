/*
 * bs_oracle.c -- plain, slow, FP64 CPU oracle for the Benchmark Streaming
 * (BS1-BS7) operations and the conjugate-gradient iteration of
 * Chalmers & Warburton, "Portable high-order finite element kernels I:
 * Streaming Operations" (arXiv 2009.10917).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  The GPU library
 * (libbs) never links, loads or calls it; the two share no source, header,
 * table or helper.  Inputs reach both sides from a separate seeded generator.
 *
 * Every routine is the literal definition, in the paper's order and
 * notation, so that it can be checked against the paper by eye: no blocking,
 * no fusion, no reordering.  The file is compiled with -ffp-contract=off, so
 * every fused multiply-add is an explicit fma() and every other product and
 * sum is rounded on its own.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *  - BS2 is y = fma(alpha, x, beta*y)                        (Table 1, BS2)
 *  - BS3/BS4 return the correctly rounded sum as far as a doubled-precision
 *    dot product (Ogita, Rump & Oishi 2005, "Dot2") gives it  (Table 1)
 *  - BS6 sums the local copies of a global node in ascending local index,
 *    starting from +0.0; a global node with no copies is 0  (eq. scatter_def)
 *  - BS7 leaves masked (id < 0) local entries untouched      (Sec. 5)
 *  - the operator is the affine-cube GLL spectral element discretisation of
 *    the Helmholtz weak form with collocated (lumped) quadrature (Sec. 2);
 *    the *_geo entry points take general trilinear hexahedra instead
 *    (eight corner vertices per element; the non-affine geometric factors
 *    that the paper's BS6/BS7 discussion mentions, Sec. 5)
 *  - CG stops when r.r <= tol^2 * (b.b)                       (Algorithm 1)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Error-free transformations (Ogita, Rump & Oishi, SIAM J. Sci. Comput.    */
/* 26(6), 2005): TwoSum (Knuth) and TwoProduct (by fma).                    */
/* ------------------------------------------------------------------------ */
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

/* Dot2: sum of x_i*y_i as if accumulated in twice the working precision,
 * then rounded once. */
static double dot2(int64_t n, const double *x, const double *y) {
  if (n <= 0) return 0.0;
  double p, s, h, r, q;
  two_prod(x[0], y[0], &p, &s);
  for (int64_t i = 1; i < n; ++i) {
    two_prod(x[i], y[i], &h, &r);
    two_sum(p, h, &p, &q);
    s = s + (q + r);
  }
  return p + s;
}

/* ------------------------------------------------------------------------ */
/* BS1-BS5 (Table 1; Listings 1-3)                                          */
/* ------------------------------------------------------------------------ */

/* BS1, vector copy: y = x. */
void bso_copy(int64_t n, const double *x, double *y) {
  for (int64_t i = 0; i < n; ++i) y[i] = x[i];
}

/* BS2, vector AXPY: y = alpha*x + beta*y, read as fma(alpha, x, beta*y). */
void bso_axpy(int64_t n, double alpha, const double *x, double beta, double *y) {
  for (int64_t i = 0; i < n; ++i) y[i] = fma(alpha, x[i], beta * y[i]);
}

/* BS3, vector norm: out[0] = x.x, out[1] = sqrt(x.x). */
void bso_norm(int64_t n, const double *x, double *out) {
  double s = dot2(n, x, x);
  out[0] = s;
  out[1] = sqrt(s);
}

/* BS4, inner product: x.y. */
double bso_dot(int64_t n, const double *x, const double *y) {
  return dot2(n, x, y);
}

/* BS5, fused CG update (Algorithm 1, steps 8-10 fused):
 *   x = x + alpha p,  r = r - alpha Ap,  returns r.r of the updated r. */
double bso_cg_update(int64_t n, double alpha, const double *p, const double *Ap,
                     double *x, double *r) {
  for (int64_t i = 0; i < n; ++i) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, Ap[i], r[i]);
  }
  return dot2(n, r, r);
}

/* ------------------------------------------------------------------------ */
/* BS6/BS7: gather and scatter (eq. scatter_def; Listings 4-5)              */
/* ------------------------------------------------------------------------ */

/* BS7, scatter q_L = Z q_G: q_L[l] = q_G[ids[l]] where ids[l] >= 0; masked
 * entries keep their previous value. */
void bso_scatter(int64_t NL, const int32_t *ids, const double *qG, double *qL) {
  for (int64_t l = 0; l < NL; ++l)
    if (ids[l] >= 0) qL[l] = qG[ids[l]];
}

/* BS6, gather q_G = Z^T q_L: q_G[g] = sum of q_L[l] over {l : ids[l] = g},
 * accumulated in ascending l from +0.0. */
void bso_gather(int64_t NL, int64_t NG, const int32_t *ids, const double *qL,
                double *qG) {
  for (int64_t g = 0; g < NG; ++g) qG[g] = 0.0;
  for (int64_t l = 0; l < NL; ++l)
    if (ids[l] >= 0) qG[ids[l]] = qG[ids[l]] + qL[l];
}

/* Valence of every global node: the diagonal of Z^T Z. */
void bso_valence(int64_t NL, int64_t NG, const int32_t *ids, int32_t *val) {
  for (int64_t g = 0; g < NG; ++g) val[g] = 0;
  for (int64_t l = 0; l < NL; ++l)
    if (ids[l] >= 0) val[ids[l]] += 1;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Lobatto-Legendre nodes, weights and differentiation matrix         */
/* (Sec. 2, eq. basis): the nodes are -1, +1 and the roots of P_N'.         */
/* ------------------------------------------------------------------------ */

/* Legendre P_N(x), P_N'(x) by the three-term recurrence
 *   (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},
 * and P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
static void legendre(int N, double x, double *PN, double *dPN) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (N == 0) { *PN = 1.0; *dPN = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *PN = p1;
  *dPN = d1;
}

/* r[0..N], w[0..N], D[(N+1)*(N+1)] row-major: D[a*(N+1)+i] = l_i'(r_a).
 * Returns 0 on success. */
int bso_gll(int N, double *r, double *w, double *D) {
  if (N < 1 || N > 32) return 1;
  const double pi = 3.14159265358979323846;
  r[0] = -1.0;
  r[N] = 1.0;
  /* interior nodes: Newton on P_N'(x) = 0 from Chebyshev-Lobatto guesses;
   * P_N'' from the Legendre equation (1-x^2) P'' = 2x P' - N(N+1) P. */
  for (int i = 1; i < N; ++i) {
    double x = -cos(pi * i / N);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(N, x, &P, &dP);
      double d2P = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
      double dx = dP / d2P;
      x -= dx;
      if (fabs(dx) <= 1e-17) break;
    }
    r[i] = x;
  }
  /* enforce the symmetry r_i = -r_{N-i} */
  for (int i = 0; i <= N / 2; ++i) {
    double s = 0.5 * (r[N - i] - r[i]);
    r[i] = -s;
    r[N - i] = s;
  }
  if (N % 2 == 0) r[N / 2] = 0.0;
  double PN[33];
  for (int i = 0; i <= N; ++i) {
    double dP;
    legendre(N, r[i], &PN[i], &dP);
    w[i] = 2.0 / (N * (N + 1.0) * PN[i] * PN[i]);
  }
  int Nq = N + 1;
  for (int a = 0; a <= N; ++a)
    for (int i = 0; i <= N; ++i) {
      double v;
      if (a != i)
        v = PN[a] / (PN[i] * (r[a] - r[i]));
      else if (a == 0)
        v = -N * (N + 1.0) / 4.0;
      else if (a == N)
        v = N * (N + 1.0) / 4.0;
      else
        v = 0.0;
      D[a * Nq + i] = v;
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Operator A = Z^T (S_L + lambda M_L) Z  (eqs. global_system,              */
/* assembled_stiff, assembled_mass).  Elements are affine cubes of side h;  */
/* element e carries a stiffness coefficient c_e (1 when coef is NULL).     */
/* Local node (i,j,k) of element e sits at l = e*Np + i + Nq*(j + Nq*k).    */
/* On element e, with u the local values and quadrature on the GLL nodes:   */
/*   (A_e u)_ijk = c_e (h/2) sum_q w_q grad l_ijk(q) . grad u(q)            */
/*               + lambda (h/2)^3 w_i w_j w_k u_ijk                         */
/* (reference gradient; the affine map contributes (2/h)^2 (h/2)^3 = h/2).  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int E, N;
  double h, lambda;
  const double *coef; /* per-element stiffness coefficient or NULL */
  const int32_t *ids; /* local -> global, length E*(N+1)^3, < 0 masked */
  int64_t NG;
  const double *verts; /* NULL: affine cubes of side h; else 24 per element */
} bso_problem;

/* ------------------------------------------------------------------------ */
/* General hexahedra.  Element e is the trilinear image of [-1,1]^3 with    */
/* corner v = vx + 2 (vy + 2 vz) (vx, vy, vz in {0, 1}) at                 */
/* verts[24 e + 3 v + d], d = x, y, z:                                      */
/*   x(r,s,t) = sum_v X_v (1 + sx r)(1 + sy s)(1 + sz t) / 8,  sx = 2vx - 1. */
/* With J = dx/dr (J[d][p] = d x_d / d r_p) at a GLL node q,                */
/*   (A_e u)_n = c_e sum_q w_q det J  (J^-T grad_r l_n)(q) . (J^-T grad_r u)(q) */
/*             + lambda w_n det J(n) u_n,                                   */
/* i.e. the reference gradient contracted with G = w_q det J J^-1 J^-T.     */
/* ------------------------------------------------------------------------ */

static void jacobian(const double *X, double r, double s, double t, double J[3][3]) {
  for (int d = 0; d < 3; ++d) J[d][0] = J[d][1] = J[d][2] = 0.0;
  for (int v = 0; v < 8; ++v) {
    const double sx = (v & 1) ? 1.0 : -1.0, sy = (v & 2) ? 1.0 : -1.0, sz = (v & 4) ? 1.0 : -1.0;
    const double dr = sx * (1.0 + sy * s) * (1.0 + sz * t) / 8.0;
    const double ds = (1.0 + sx * r) * sy * (1.0 + sz * t) / 8.0;
    const double dt = (1.0 + sx * r) * (1.0 + sy * s) * sz / 8.0;
    for (int d = 0; d < 3; ++d) {
      J[d][0] += X[3 * v + d] * dr;
      J[d][1] += X[3 * v + d] * ds;
      J[d][2] += X[3 * v + d] * dt;
    }
  }
}

static double det3(double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* G[p][q] = wq det J sum_d Jinv[p][d] Jinv[q][d], Jinv = J^-1 by cofactors. */
static double metric(double J[3][3], double wq, double G[3][3]) {
  const double det = det3(J);
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) {
      double v = 0.0;
      for (int d = 0; d < 3; ++d) v += inv[p][d] * inv[q][d];
      G[p][q] = wq * det * v;
    }
  return det;
}

static void element_apply_geo(const bso_problem *P, const double *r, const double *w,
                              const double *D, int e, const double *u, double *Au,
                              double *ur, double *us, double *ut) {
  const int N = P->N, Nq = N + 1;
  const double ce = P->coef ? P->coef[e] : 1.0;
  const double *X = P->verts + (int64_t)e * 24;
  double J[3][3], G[3][3];
#define IDX(i, j, k) ((i) + Nq * ((j) + Nq * (k)))
  for (int c = 0; c < Nq; ++c)
    for (int b = 0; b < Nq; ++b)
      for (int a = 0; a < Nq; ++a) {
        double dr = 0.0, ds = 0.0, dt = 0.0;
        for (int n = 0; n < Nq; ++n) {
          dr = fma(D[a * Nq + n], u[IDX(n, b, c)], dr);
          ds = fma(D[b * Nq + n], u[IDX(a, n, c)], ds);
          dt = fma(D[c * Nq + n], u[IDX(a, b, n)], dt);
        }
        jacobian(X, r[a], r[b], r[c], J);
        metric(J, w[a] * w[b] * w[c], G);
        ur[IDX(a, b, c)] = G[0][0] * dr + G[0][1] * ds + G[0][2] * dt;
        us[IDX(a, b, c)] = G[1][0] * dr + G[1][1] * ds + G[1][2] * dt;
        ut[IDX(a, b, c)] = G[2][0] * dr + G[2][1] * ds + G[2][2] * dt;
      }
  for (int k = 0; k < Nq; ++k)
    for (int j = 0; j < Nq; ++j)
      for (int i = 0; i < Nq; ++i) {
        double s = 0.0;
        for (int n = 0; n < Nq; ++n) {
          s = fma(D[n * Nq + i], ur[IDX(n, j, k)], s);
          s = fma(D[n * Nq + j], us[IDX(i, n, k)], s);
          s = fma(D[n * Nq + k], ut[IDX(i, j, n)], s);
        }
        jacobian(X, r[i], r[j], r[k], J);
        const double mass = (w[i] * w[j] * w[k]) * det3(J) * u[IDX(i, j, k)];
        Au[IDX(i, j, k)] = fma(ce, s, P->lambda * mass);
      }
#undef IDX
}

static void element_apply(const bso_problem *P, const double *r, const double *w,
                          const double *D, int e, const double *u, double *Au,
                          double *ur, double *us, double *ut) {
  if (P->verts) {
    element_apply_geo(P, r, w, D, e, u, Au, ur, us, ut);
    return;
  }
  const int N = P->N, Nq = N + 1;
  const double ce = P->coef ? P->coef[e] : 1.0;
  const double g = 0.5 * P->h;          /* (h/2): stiffness geometric factor */
  const double m = g * g * g;           /* (h/2)^3: mass geometric factor     */
#define IDX(i, j, k) ((i) + Nq * ((j) + Nq * (k)))
  /* reference gradient of u at every quadrature node (a,b,c) */
  for (int c = 0; c < Nq; ++c)
    for (int b = 0; b < Nq; ++b)
      for (int a = 0; a < Nq; ++a) {
        double dr = 0.0, ds = 0.0, dt = 0.0;
        for (int n = 0; n < Nq; ++n) {
          dr = fma(D[a * Nq + n], u[IDX(n, b, c)], dr);
          ds = fma(D[b * Nq + n], u[IDX(a, n, c)], ds);
          dt = fma(D[c * Nq + n], u[IDX(a, b, n)], dt);
        }
        double wq = w[a] * w[b] * w[c];
        ur[IDX(a, b, c)] = wq * dr;
        us[IDX(a, b, c)] = wq * ds;
        ut[IDX(a, b, c)] = wq * dt;
      }
  /* test with grad l_ijk: sum over quadrature nodes of D^T applied */
  for (int k = 0; k < Nq; ++k)
    for (int j = 0; j < Nq; ++j)
      for (int i = 0; i < Nq; ++i) {
        double s = 0.0;
        for (int n = 0; n < Nq; ++n) {
          s = fma(D[n * Nq + i], ur[IDX(n, j, k)], s);
          s = fma(D[n * Nq + j], us[IDX(i, n, k)], s);
          s = fma(D[n * Nq + k], ut[IDX(i, j, n)], s);
        }
        double mass = m * (w[i] * w[j] * w[k]) * u[IDX(i, j, k)];
        Au[IDX(i, j, k)] = fma(ce * g, s, P->lambda * mass);
      }
#undef IDX
}

static int apply_A(const bso_problem *P, const double *p, double *Ap) {
  const int N = P->N, Nq = N + 1, Np = Nq * Nq * Nq;
  double r[33], w[33], D[33 * 33];
  if (bso_gll(N, r, w, D)) return 1;
  double *u = malloc(sizeof(double) * 5 * Np);
  if (!u) return 2;
  double *Au = u + Np, *ur = Au + Np, *us = ur + Np, *ut = us + Np;
  for (int64_t gI = 0; gI < P->NG; ++gI) Ap[gI] = 0.0;
  for (int e = 0; e < P->E; ++e) {
    const int32_t *id = P->ids + (int64_t)e * Np;
    for (int l = 0; l < Np; ++l) u[l] = id[l] >= 0 ? p[id[l]] : 0.0; /* Z p */
    element_apply(P, r, w, D, e, u, Au, ur, us, ut);
    for (int l = 0; l < Np; ++l) /* Z^T, ascending local index */
      if (id[l] >= 0) Ap[id[l]] = Ap[id[l]] + Au[l];
  }
  free(u);
  return 0;
}

int bso_apply_A(int E, int N, double h, double lambda, const double *coef,
                const int32_t *ids, int64_t NG, const double *p, double *Ap) {
  bso_problem P = {E, N, h, lambda, coef, ids, NG};
  return apply_A(&P, p, Ap);
}

/* Element-local operator only (no Z, no Z^T): uL -> A_L uL. */
int bso_apply_local(int E, int N, double h, double lambda, const double *coef,
                    const double *uL, double *AuL) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  double r[33], w[33], D[33 * 33];
  if (bso_gll(N, r, w, D)) return 1;
  bso_problem P = {E, N, h, lambda, coef, NULL, 0};
  double *tmp = malloc(sizeof(double) * 3 * Np);
  if (!tmp) return 2;
  for (int e = 0; e < E; ++e)
    element_apply(&P, r, w, D, e, uL + (int64_t)e * Np, AuL + (int64_t)e * Np, tmp,
                  tmp + Np, tmp + 2 * Np);
  free(tmp);
  return 0;
}

/* diag(A) = Z^T diag(A_L), with
 *   diag(S_e)_ijk = (h/2) sum_q w_q |grad l_ijk(q)|^2
 *                 = (h/2) (K_ii w_j w_k + w_i K_jj w_k + w_i w_j K_kk),
 *   K_ii = sum_a w_a D_ai^2. */
int bso_diag_A(int E, int N, double h, double lambda, const double *coef,
               const int32_t *ids, int64_t NG, double *diag) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  double r[33], w[33], D[33 * 33], K[33];
  if (bso_gll(N, r, w, D)) return 1;
  for (int i = 0; i < Nq; ++i) {
    double s = 0.0;
    for (int a = 0; a < Nq; ++a) s = fma(w[a] * D[a * Nq + i], D[a * Nq + i], s);
    K[i] = s;
  }
  const double g = 0.5 * h, m = g * g * g;
  for (int64_t gI = 0; gI < NG; ++gI) diag[gI] = 0.0;
  for (int e = 0; e < E; ++e) {
    const double ce = coef ? coef[e] : 1.0;
    for (int k = 0; k < Nq; ++k)
      for (int j = 0; j < Nq; ++j)
        for (int i = 0; i < Nq; ++i) {
          int l = i + Nq * (j + Nq * k);
          int32_t id = ids[(int64_t)e * Np + l];
          if (id < 0) continue;
          double s = K[i] * w[j] * w[k] + w[i] * K[j] * w[k] + w[i] * w[j] * K[k];
          double v = ce * g * s + lambda * m * (w[i] * w[j] * w[k]);
          diag[id] = diag[id] + v;
        }
  }
  return 0;
}

/* The general-hexahedron operator (see jacobian above). */
int bso_apply_A_geo(int E, int N, double lambda, const double *coef, const double *verts,
                    const int32_t *ids, int64_t NG, const double *p, double *Ap) {
  bso_problem P = {E, N, 1.0, lambda, coef, ids, NG, verts};
  return apply_A(&P, p, Ap);
}

int bso_apply_local_geo(int E, int N, double lambda, const double *coef, const double *verts,
                        const double *uL, double *AuL) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  double r[33], w[33], D[33 * 33];
  if (bso_gll(N, r, w, D)) return 1;
  bso_problem P = {E, N, 1.0, lambda, coef, NULL, 0, verts};
  double *tmp = malloc(sizeof(double) * 3 * Np);
  if (!tmp) return 2;
  for (int e = 0; e < E; ++e)
    element_apply(&P, r, w, D, e, uL + (int64_t)e * Np, AuL + (int64_t)e * Np, tmp,
                  tmp + Np, tmp + 2 * Np);
  free(tmp);
  return 0;
}

/* diag(A) = Z^T diag(A_L), each diagonal entry of A_e read off A_e applied
 * to the unit vector of its node. */
int bso_diag_A_geo(int E, int N, double lambda, const double *coef, const double *verts,
                   const int32_t *ids, int64_t NG, double *diag) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  double r[33], w[33], D[33 * 33];
  if (bso_gll(N, r, w, D)) return 1;
  bso_problem P = {E, N, 1.0, lambda, coef, ids, NG, verts};
  double *buf = malloc(sizeof(double) * 5 * Np);
  if (!buf) return 2;
  double *unit = buf, *col = buf + Np;
  for (int64_t gI = 0; gI < NG; ++gI) diag[gI] = 0.0;
  for (int e = 0; e < E; ++e)
    for (int l = 0; l < Np; ++l) {
      const int32_t id = ids[(int64_t)e * Np + l];
      if (id < 0) continue;
      for (int m = 0; m < Np; ++m) unit[m] = 0.0;
      unit[l] = 1.0;
      element_apply(&P, r, w, D, e, unit, col, col + Np, col + 2 * Np, col + 3 * Np);
      diag[id] = diag[id] + col[l];
    }
  free(buf);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Training pairs of the learned element preconditioner (no counterpart in  */
/* the paper; the definition this project chose).  For a global residual r  */
/* and element e, with u = D^-1 r (D = diag A) read through the map:        */
/*   rms   = sqrt(mean over the element's Np nodes of u^2)                  */
/*   e_I   = A_II^-1 r_I : the element-interior error, i.e. the correction  */
/*           that zeroes the residual on the element's interior nodes       */
/*           (1 <= i,j,k <= N-1, not masked) with its other nodes held;     */
/*           A_II is the interior block of c_e S_e + lambda M_e             */
/*   X     = s u / rms,  T = s (e_I - u_I) / rms on interior nodes, 0 else  */
/* with s = -1 for odd pair index when negate_odd (the sign-flipped pair    */
/* (-r, -e) is as valid as (r, e)), else s = 1; rms = 0 gives zero rows.    */
/* A_II is formed column by column with element_apply and solved by a       */
/* dense Cholesky factorisation.  Returns 0, 1 on a bad degree, 2 on an     */
/* allocation failure, 3 if an A_II is not positive definite.               */
/* ------------------------------------------------------------------------ */
int bso_interior_pairs(int E, int N, double h, double lambda, const double *coef,
                       const int32_t *ids, int64_t NG, const double *rG, int64_t count,
                       const int32_t *elems, int negate_odd, float *X, float *T) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  double r[33], w[33], D[33 * 33];
  if (bso_gll(N, r, w, D)) return 1;
  bso_problem P = {E, N, h, lambda, coef, ids, NG};
  double *dg = malloc(sizeof(double) * (NG > 0 ? NG : 1));
  double *buf = malloc(sizeof(double) * ((size_t)Np * Np + 7 * (size_t)Np));
  int *I = malloc(sizeof(int) * Np);
  if (!dg || !buf || !I) { free(dg); free(buf); free(I); return 2; }
  double *Aii = buf, *u = Aii + (size_t)Np * Np, *unit = u + Np, *col = unit + Np,
         *t1 = col + Np, *t2 = t1 + Np, *t3 = t2 + Np, *y = t3 + Np;
  bso_diag_A(E, N, h, lambda, coef, ids, NG, dg);
  int rc = 0;
  for (int64_t q = 0; q < count && !rc; ++q) {
    const int e = elems[q];
    const int32_t *id = ids + (int64_t)e * Np;
    const double s = (negate_odd && (q & 1)) ? -1.0 : 1.0;
    double ss = 0.0;
    for (int l = 0; l < Np; ++l) {
      u[l] = id[l] >= 0 ? rG[id[l]] / dg[id[l]] : 0.0;
      ss += u[l] * u[l];
    }
    const double rms = sqrt(ss / Np);
    float *xo = X + q * Np, *to = T + q * Np;
    for (int l = 0; l < Np; ++l) xo[l] = to[l] = 0.0f;
    if (!(rms > 0.0)) continue;
    int nI = 0;
    for (int k = 1; k < N; ++k)
      for (int j = 1; j < N; ++j)
        for (int i = 1; i < N; ++i) {
          const int l = i + Nq * (j + Nq * k);
          if (id[l] >= 0) I[nI++] = l;
        }
    /* A_II, column c = interior rows of A_e applied to unit vector c */
    for (int c = 0; c < nI; ++c) {
      for (int l = 0; l < Np; ++l) unit[l] = 0.0;
      unit[I[c]] = 1.0;
      element_apply(&P, r, w, D, e, unit, col, t1, t2, t3);
      for (int a = 0; a < nI; ++a) Aii[a * nI + c] = col[I[a]];
    }
    /* Cholesky A_II = L L^T in place (lower triangle) */
    for (int c = 0; c < nI && !rc; ++c) {
      double d = Aii[c * nI + c];
      for (int k = 0; k < c; ++k) d -= Aii[c * nI + k] * Aii[c * nI + k];
      if (!(d > 0.0)) { rc = 3; break; }
      d = sqrt(d);
      Aii[c * nI + c] = d;
      for (int a = c + 1; a < nI; ++a) {
        double v = Aii[a * nI + c];
        for (int k = 0; k < c; ++k) v -= Aii[a * nI + k] * Aii[c * nI + k];
        Aii[a * nI + c] = v / d;
      }
    }
    if (rc) break;
    /* forward then backward substitution on r_I */
    for (int a = 0; a < nI; ++a) {
      double v = rG[id[I[a]]];
      for (int k = 0; k < a; ++k) v -= Aii[a * nI + k] * y[k];
      y[a] = v / Aii[a * nI + a];
    }
    for (int a = nI - 1; a >= 0; --a) {
      double v = y[a];
      for (int k = a + 1; k < nI; ++k) v -= Aii[k * nI + a] * y[k];
      y[a] = v / Aii[a * nI + a];
    }
    for (int l = 0; l < Np; ++l) xo[l] = (float)(s * u[l] / rms);
    for (int a = 0; a < nI; ++a) to[I[a]] = (float)(s * (y[a] - u[I[a]]) / rms);
  }
  free(dg); free(buf); free(I);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradients (Algorithm 1) on A u = b.                            */
/* x holds the initial guess on entry and the solution on exit.             */
/* Iterates until r.r <= tol^2 (b.b) or maxit; with fixed_iters != 0 runs   */
/* exactly maxit iterations.  Optional histories (length >= maxit+1) record */
/* alpha_j, beta_j and r_j.r_j (hist_rr[0] is r_0.r_0).                     */
/* Returns the iteration count, or -1 on a breakdown (p.Ap <= 0 or not      */
/* finite), -2 on an allocation failure.                                    */
/* ------------------------------------------------------------------------ */
static int cg_run(const bso_problem *Pp, const double *b, double *x, double tol, int maxit,
                  int fixed_iters, double *hist_alpha, double *hist_beta, double *hist_rr) {
  const bso_problem P = *Pp;
  const int64_t NG = P.NG;
  double *r = malloc(sizeof(double) * 3 * NG);
  if (!r) return -2;
  double *p = r + NG, *Ap = p + NG;
  /* r_0 = b - A x */
  if (apply_A(&P, x, Ap)) { free(r); return -2; }
  for (int64_t i = 0; i < NG; ++i) r[i] = b[i] - Ap[i];
  /* p = r */
  for (int64_t i = 0; i < NG; ++i) p[i] = r[i];
  double rr = dot2(NG, r, r);
  const double eps = tol * tol * dot2(NG, b, b);
  if (hist_rr) hist_rr[0] = rr;
  int j = 0;
  while (j < maxit && (fixed_iters || rr > eps)) {
    apply_A(&P, p, Ap);
    double pAp = dot2(NG, p, Ap);
    if (!(pAp > 0.0) || !isfinite(pAp)) { free(r); return -1; }
    double alpha = rr / pAp;                                  /* step 7  */
    double rr_new = bso_cg_update(NG, alpha, p, Ap, x, r);    /* 8-10    */
    double beta = rr_new / rr;                                /* step 10 */
    for (int64_t i = 0; i < NG; ++i) p[i] = fma(1.0, r[i], beta * p[i]); /* 11 */
    rr = rr_new;
    if (hist_alpha) hist_alpha[j] = alpha;
    if (hist_beta) hist_beta[j] = beta;
    if (hist_rr) hist_rr[j + 1] = rr;
    ++j;
  }
  free(r);
  return j;
}

int bso_cg(int E, int N, double h, double lambda, const double *coef,
           const int32_t *ids, int64_t NG, const double *b, double *x, double tol,
           int maxit, int fixed_iters, double *hist_alpha, double *hist_beta,
           double *hist_rr) {
  bso_problem P = {E, N, h, lambda, coef, ids, NG, NULL};
  return cg_run(&P, b, x, tol, maxit, fixed_iters, hist_alpha, hist_beta, hist_rr);
}

int bso_cg_geo(int E, int N, double lambda, const double *coef, const double *verts,
               const int32_t *ids, int64_t NG, const double *b, double *x, double tol,
               int maxit, int fixed_iters, double *hist_alpha, double *hist_beta,
               double *hist_rr) {
  bso_problem P = {E, N, 1.0, lambda, coef, ids, NG, verts};
  return cg_run(&P, b, x, tol, maxit, fixed_iters, hist_alpha, hist_beta, hist_rr);
}

/* Jacobi-preconditioned CG: Algorithm 1 with z = diag(A)^{-1} r, alpha =
 * r.z / p.Ap, beta = r_{j+1}.z_{j+1} / r_j.z_j, p = z + beta p.  Stops on the
 * unpreconditioned r.r <= tol^2 (b.b). */
static int pcg_run(const bso_problem *Pp, const double *b, double *x, double tol, int maxit,
                   double *hist_rr) {
  const bso_problem P = *Pp;
  const int64_t NG = P.NG;
  double *r = malloc(sizeof(double) * 5 * NG);
  if (!r) return -2;
  double *p = r + NG, *Ap = p + NG, *z = Ap + NG, *dg = z + NG;
  if (P.verts)
    bso_diag_A_geo(P.E, P.N, P.lambda, P.coef, P.verts, P.ids, NG, dg);
  else
    bso_diag_A(P.E, P.N, P.h, P.lambda, P.coef, P.ids, NG, dg);
  apply_A(&P, x, Ap);
  for (int64_t i = 0; i < NG; ++i) r[i] = b[i] - Ap[i];
  for (int64_t i = 0; i < NG; ++i) z[i] = r[i] / dg[i];
  for (int64_t i = 0; i < NG; ++i) p[i] = z[i];
  double rz = dot2(NG, r, z), rr = dot2(NG, r, r);
  const double eps = tol * tol * dot2(NG, b, b);
  if (hist_rr) hist_rr[0] = rr;
  int j = 0;
  while (j < maxit && rr > eps) {
    apply_A(&P, p, Ap);
    double pAp = dot2(NG, p, Ap);
    if (!(pAp > 0.0) || !isfinite(pAp)) { free(r); return -1; }
    double alpha = rz / pAp;
    rr = bso_cg_update(NG, alpha, p, Ap, x, r);
    for (int64_t i = 0; i < NG; ++i) z[i] = r[i] / dg[i];
    double rz_new = dot2(NG, r, z);
    double beta = rz_new / rz;
    for (int64_t i = 0; i < NG; ++i) p[i] = fma(1.0, z[i], beta * p[i]);
    rz = rz_new;
    ++j;
    if (hist_rr) hist_rr[j] = rr;
  }
  free(r);
  return j;
}

int bso_pcg_jacobi(int E, int N, double h, double lambda, const double *coef,
                   const int32_t *ids, int64_t NG, const double *b, double *x,
                   double tol, int maxit, double *hist_rr) {
  bso_problem P = {E, N, h, lambda, coef, ids, NG, NULL};
  return pcg_run(&P, b, x, tol, maxit, hist_rr);
}

int bso_pcg_jacobi_geo(int E, int N, double lambda, const double *coef, const double *verts,
                       const int32_t *ids, int64_t NG, const double *b, double *x,
                       double tol, int maxit, double *hist_rr) {
  bso_problem P = {E, N, 1.0, lambda, coef, ids, NG, verts};
  return pcg_run(&P, b, x, tol, maxit, hist_rr);
}

/* ------------------------------------------------------------------------ */
/* Block-Jacobi PCG (the exact form of the learned preconditioner's map):   */
/* z = M^-1 r with, for every element e whose interior local nodes I_e are  */
/* all unmasked and held by e alone (valence 1), the block solved exactly,  */
/*   z[ids(I_e)] = A_II^-1 r[ids(I_e)],  A_II = rows/cols I_e of            */
/*   c_e S_e + lambda M_e (Cholesky, factored once per element),            */
/* and z_g = r_g / diag(A)_g at every other node.  Algorithm 1 with z.      */
/* ------------------------------------------------------------------------ */
int bso_pcg_block_jacobi(int E, int N, double h, double lambda, const double *coef,
                         const int32_t *ids, int64_t NG, const double *b, double *x,
                         double tol, int maxit, double *hist_rr) {
  const int Nq = N + 1, Np = Nq * Nq * Nq, nImax = (N - 1) * (N - 1) * (N - 1);
  double gr[33], gw[33], gD[33 * 33];
  if (N < 2 || bso_gll(N, gr, gw, gD)) return -3;
  bso_problem P = {E, N, h, lambda, coef, ids, NG, NULL};
  double *vec = malloc(sizeof(double) * 5 * (NG > 0 ? NG : 1));
  double *L = malloc(sizeof(double) * (size_t)E * nImax * nImax + 1);
  int *I = malloc(sizeof(int) * (size_t)E * nImax + 1), *nI = malloc(sizeof(int) * (E + 1));
  int *val = malloc(sizeof(int) * (NG > 0 ? NG : 1));
  double *tmp = malloc(sizeof(double) * 6 * Np);
  if (!vec || !L || !I || !nI || !val || !tmp) {
    free(vec); free(L); free(I); free(nI); free(val); free(tmp);
    return -2;
  }
  double *r = vec, *p = r + NG, *Ap = p + NG, *z = Ap + NG, *dg = z + NG;
  double *unit = tmp, *col = unit + Np, *t1 = col + Np, *t2 = t1 + Np, *t3 = t2 + Np,
         *y = t3 + Np;
  bso_diag_A(E, N, h, lambda, coef, ids, NG, dg);
  bso_valence((int64_t)E * Np, NG, ids, val);
  int rc = 0;
  for (int e = 0; e < E && !rc; ++e) {
    const int32_t *id = ids + (int64_t)e * Np;
    int *Ie = I + (size_t)e * nImax;
    double *Le = L + (size_t)e * nImax * nImax;
    int n = 0, all = 1;
    for (int k = 1; k < N; ++k)
      for (int j = 1; j < N; ++j)
        for (int i = 1; i < N; ++i) {
          const int l = i + Nq * (j + Nq * k);
          if (id[l] >= 0 && val[id[l]] == 1)
            Ie[n++] = l;
          else
            all = 0;
        }
    if (!all) n = 0;  /* the interior is not a block of A: Jacobi there */
    nI[e] = n;
    for (int c = 0; c < n; ++c) {  /* column c of A_II */
      for (int l = 0; l < Np; ++l) unit[l] = 0.0;
      unit[Ie[c]] = 1.0;
      element_apply(&P, gr, gw, gD, e, unit, col, t1, t2, t3);
      for (int a = 0; a < n; ++a) Le[a * n + c] = col[Ie[a]];
    }
    for (int c = 0; c < n && !rc; ++c) {  /* A_II = L L^T */
      double d = Le[c * n + c];
      for (int k = 0; k < c; ++k) d -= Le[c * n + k] * Le[c * n + k];
      if (!(d > 0.0)) { rc = -4; break; }
      d = sqrt(d);
      Le[c * n + c] = d;
      for (int a = c + 1; a < n; ++a) {
        double v = Le[a * n + c];
        for (int k = 0; k < c; ++k) v -= Le[a * n + k] * Le[c * n + k];
        Le[a * n + c] = v / d;
      }
    }
  }
  /* z = M^-1 r */
#define BJ_APPLY()                                                          \
  do {                                                                      \
    for (int64_t g = 0; g < NG; ++g) z[g] = r[g] / dg[g];                   \
    for (int e = 0; e < E; ++e) {                                           \
      const int32_t *id = ids + (int64_t)e * Np;                            \
      const int *Ie = I + (size_t)e * nImax, n = nI[e];                     \
      const double *Le = L + (size_t)e * nImax * nImax;                     \
      for (int a = 0; a < n; ++a) {                                         \
        double v = r[id[Ie[a]]];                                            \
        for (int k = 0; k < a; ++k) v -= Le[a * n + k] * y[k];              \
        y[a] = v / Le[a * n + a];                                           \
      }                                                                     \
      for (int a = n - 1; a >= 0; --a) {                                    \
        double v = y[a];                                                    \
        for (int k = a + 1; k < n; ++k) v -= Le[k * n + a] * y[k];          \
        y[a] = v / Le[a * n + a];                                           \
      }                                                                     \
      for (int a = 0; a < n; ++a) z[id[Ie[a]]] = y[a];                      \
    }                                                                       \
  } while (0)
  int j = 0;
  if (!rc) {
    apply_A(&P, x, Ap);
    for (int64_t g = 0; g < NG; ++g) r[g] = b[g] - Ap[g];
    BJ_APPLY();
    for (int64_t g = 0; g < NG; ++g) p[g] = z[g];
    double rz = dot2(NG, r, z), rr = dot2(NG, r, r);
    const double eps = tol * tol * dot2(NG, b, b);
    if (hist_rr) hist_rr[0] = rr;
    while (j < maxit && rr > eps) {
      apply_A(&P, p, Ap);
      const double pAp = dot2(NG, p, Ap);
      if (!(pAp > 0.0) || !isfinite(pAp)) { rc = -1; break; }
      const double alpha = rz / pAp;
      rr = bso_cg_update(NG, alpha, p, Ap, x, r);
      BJ_APPLY();
      const double rz_new = dot2(NG, r, z);
      const double beta = rz_new / rz;
      for (int64_t g = 0; g < NG; ++g) p[g] = fma(1.0, z[g], beta * p[g]);
      rz = rz_new;
      ++j;
      if (hist_rr) hist_rr[j] = rr;
    }
  }
#undef BJ_APPLY
  free(vec); free(L); free(I); free(nI); free(val); free(tmp);
  return rc ? rc : j;
}

/* ------------------------------------------------------------------------ */
/* FP32-storage CG inside an FP64 iterative-refinement loop.                */
/* Outer (FP64): r = b - A x; stop when ||r|| <= outer_tol ||b||; solve     */
/* A d = r approximately in FP32; x = x + d.                                */
/* Inner (Algorithm 1 on A d = r): vectors and the operator in float;       */
/* dot products of float vectors accumulated in double and the scalars     */
/* alpha, beta formed in double, then rounded to float for the updates.     */
/* Stops at d-residual <= inner_tol * ||r|| or inner_maxit.                 */
/* Returns the total inner iteration count; *outer gets the outer count and */
/* *relres the final FP64 true relative residual.                           */
/* ------------------------------------------------------------------------ */
static double dotf(int64_t n, const float *x, const float *y) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = fma((double)x[i], (double)y[i], s);
  return s;
}

static void element_apply_f32(int N, const float *w, const float *D, float g,
                              float m, float ce, float lambda, const float *u,
                              float *Au, float *ur, float *us, float *ut) {
  const int Nq = N + 1;
#define IDX(i, j, k) ((i) + Nq * ((j) + Nq * (k)))
  for (int c = 0; c < Nq; ++c)
    for (int b = 0; b < Nq; ++b)
      for (int a = 0; a < Nq; ++a) {
        float dr = 0.f, ds = 0.f, dt = 0.f;
        for (int n = 0; n < Nq; ++n) {
          dr = fmaf(D[a * Nq + n], u[IDX(n, b, c)], dr);
          ds = fmaf(D[b * Nq + n], u[IDX(a, n, c)], ds);
          dt = fmaf(D[c * Nq + n], u[IDX(a, b, n)], dt);
        }
        float wq = w[a] * w[b] * w[c];
        ur[IDX(a, b, c)] = wq * dr;
        us[IDX(a, b, c)] = wq * ds;
        ut[IDX(a, b, c)] = wq * dt;
      }
  for (int k = 0; k < Nq; ++k)
    for (int j = 0; j < Nq; ++j)
      for (int i = 0; i < Nq; ++i) {
        float s = 0.f;
        for (int n = 0; n < Nq; ++n) {
          s = fmaf(D[n * Nq + i], ur[IDX(n, j, k)], s);
          s = fmaf(D[n * Nq + j], us[IDX(i, n, k)], s);
          s = fmaf(D[n * Nq + k], ut[IDX(i, j, n)], s);
        }
        float mass = m * (w[i] * w[j] * w[k]) * u[IDX(i, j, k)];
        Au[IDX(i, j, k)] = fmaf(ce * g, s, lambda * mass);
      }
#undef IDX
}

static void apply_A_f32(const bso_problem *P, const float *w, const float *D,
                        const float *p, float *Ap, float *buf) {
  const int N = P->N, Nq = N + 1, Np = Nq * Nq * Nq;
  float *u = buf, *Au = u + Np, *ur = Au + Np, *us = ur + Np, *ut = us + Np;
  const float g = (float)(0.5 * P->h), m = (float)(0.125 * P->h * P->h * P->h);
  for (int64_t gI = 0; gI < P->NG; ++gI) Ap[gI] = 0.f;
  for (int e = 0; e < P->E; ++e) {
    const int32_t *id = P->ids + (int64_t)e * Np;
    for (int l = 0; l < Np; ++l) u[l] = id[l] >= 0 ? p[id[l]] : 0.f;
    element_apply_f32(N, w, D, g, m, P->coef ? (float)P->coef[e] : 1.f,
                      (float)P->lambda, u, Au, ur, us, ut);
    for (int l = 0; l < Np; ++l)
      if (id[l] >= 0) Ap[id[l]] = Ap[id[l]] + Au[l];
  }
}

int bso_cg_ir_f32(int E, int N, double h, double lambda, const double *coef,
                  const int32_t *ids, int64_t NG, const double *b, double *x,
                  double outer_tol, int outer_maxit, double inner_tol,
                  int inner_maxit, int *outer, double *relres) {
  bso_problem P = {E, N, h, lambda, coef, ids, NG};
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  double rq[33], wq[33], Dq[33 * 33];
  float w[33], D[33 * 33];
  if (bso_gll(N, rq, wq, Dq)) return -2;
  for (int i = 0; i < Nq; ++i) w[i] = (float)wq[i];
  for (int i = 0; i < Nq * Nq; ++i) D[i] = (float)Dq[i];
  double *r = malloc(sizeof(double) * 2 * NG);
  float *fb = malloc(sizeof(float) * (5 * NG + 5 * Np));
  if (!r || !fb) { free(r); free(fb); return -2; }
  double *Ax = r + NG;
  float *d = fb, *rf = d + NG, *pf = rf + NG, *Apf = pf + NG, *rs = Apf + NG;
  float *buf = rs + NG;
  (void)rs;
  const double bnorm = sqrt(dot2(NG, b, b));
  int total = 0, k = 0;
  double res = 0.0;
  for (;;) {
    apply_A(&P, x, Ax);
    for (int64_t i = 0; i < NG; ++i) r[i] = b[i] - Ax[i];
    res = sqrt(dot2(NG, r, r));
    if (res <= outer_tol * bnorm || k >= outer_maxit) break;
    /* inner FP32 CG on A d = r, d_0 = 0 */
    for (int64_t i = 0; i < NG; ++i) {
      d[i] = 0.f;
      rf[i] = (float)r[i];
      pf[i] = rf[i];
    }
    double rr = dotf(NG, rf, rf);
    const double eps = inner_tol * inner_tol * rr;
    int j = 0;
    while (j < inner_maxit && rr > eps) {
      apply_A_f32(&P, w, D, pf, Apf, buf);
      double pAp = dotf(NG, pf, Apf);
      if (!(pAp > 0.0) || !isfinite(pAp)) break;
      float alpha = (float)(rr / pAp);
      for (int64_t i = 0; i < NG; ++i) {
        d[i] = fmaf(alpha, pf[i], d[i]);
        rf[i] = fmaf(-alpha, Apf[i], rf[i]);
      }
      double rr_new = dotf(NG, rf, rf);
      float beta = (float)(rr_new / rr);
      for (int64_t i = 0; i < NG; ++i) pf[i] = fmaf(1.f, rf[i], beta * pf[i]);
      rr = rr_new;
      ++j;
    }
    total += j;
    for (int64_t i = 0; i < NG; ++i) x[i] = x[i] + (double)d[i];
    ++k;
  }
  if (outer) *outer = k;
  if (relres) *relres = bnorm > 0.0 ? res / bnorm : res;
  free(r);
  free(fb);
  return total;
}

/* ------------------------------------------------------------------------ */
/* The CSR form of Z^T (Sec. 5, Listing 4), by its definition:              */
/* rowStarts[g] = #{l : 0 <= ids[l] < g}; colIds lists, row by row, the     */
/* local indices l with ids[l] = g in ascending order.                      */
/* ------------------------------------------------------------------------ */
void bso_csr(int64_t NL, int64_t NG, const int32_t *ids, int32_t *row_starts,
             int32_t *col_ids) {
  for (int64_t g = 0; g <= NG; ++g) row_starts[g] = 0;
  for (int64_t l = 0; l < NL; ++l)
    if (ids[l] >= 0) row_starts[ids[l] + 1] += 1;
  for (int64_t g = 0; g < NG; ++g) row_starts[g + 1] += row_starts[g];
  /* rows in order, each row's l ascending: one stable bucket pass */
  int32_t *next = malloc(sizeof(int32_t) * (size_t)(NG > 0 ? NG : 1));
  if (!next) return;
  for (int64_t g = 0; g < NG; ++g) next[g] = row_starts[g];
  for (int64_t l = 0; l < NL; ++l)
    if (ids[l] >= 0) col_ids[next[ids[l]]++] = (int32_t)l;
  free(next);
}

/* ------------------------------------------------------------------------ */
/* FP32-storage twins of BS2, BS5, BS6, BS7: the same definitions with      */
/* float values and fmaf; the r.r of BS5 is the Dot2 sum of the updated     */
/* float values taken as doubles (their products are exact in double).     */
/* ------------------------------------------------------------------------ */
void bso_axpy_f32(int64_t n, float alpha, const float *x, float beta, float *y) {
  for (int64_t i = 0; i < n; ++i) y[i] = fmaf(alpha, x[i], beta * y[i]);
}

double bso_dot_f32(int64_t n, const float *x, const float *y) {
  if (n <= 0) return 0.0;
  double p, s, h, r, q;
  two_prod((double)x[0], (double)y[0], &p, &s);
  for (int64_t i = 1; i < n; ++i) {
    two_prod((double)x[i], (double)y[i], &h, &r);
    two_sum(p, h, &p, &q);
    s = s + (q + r);
  }
  return p + s;
}

double bso_cg_update_f32(int64_t n, float alpha, const float *p, const float *Ap,
                         float *x, float *r) {
  for (int64_t i = 0; i < n; ++i) {
    x[i] = fmaf(alpha, p[i], x[i]);
    r[i] = fmaf(-alpha, Ap[i], r[i]);
  }
  return bso_dot_f32(n, r, r);
}

void bso_scatter_f32(int64_t NL, const int32_t *ids, const float *qG, float *qL) {
  for (int64_t l = 0; l < NL; ++l)
    if (ids[l] >= 0) qL[l] = qG[ids[l]];
}

void bso_gather_f32(int64_t NL, int64_t NG, const int32_t *ids, const float *qL,
                    float *qG) {
  for (int64_t g = 0; g < NG; ++g) qG[g] = 0.0f;
  for (int64_t l = 0; l < NL; ++l)
    if (ids[l] >= 0) qG[ids[l]] = qG[ids[l]] + qL[l];
}
