/*
 * mlp_oracle.c -- FP64 CPU oracle of the learned element preconditioner:
 * a two-layer MLP without biases, its MSE loss and gradients, Adam, and
 * flexible PCG (Polak-Ribiere beta) with the MLP correction and a Jacobi
 * fallback.  TEST INFRASTRUCTURE ONLY (see bs_oracle.c).
 *
 * The paper has no learned part; these are the definitions this project
 * chose (listed in the design notes):
 *   MLP:  y = W2 relu(W1 x),  W1: H x D,  W2: D x H (row-major, no biases)
 *   Precision modes (prec) of the network's products:
 *     0  FP64 products of the float values;
 *     1  BF16: x, W1, W2 and the hidden activations rounded to bfloat16
 *        (round to nearest even from the float value) where the GPU rounds
 *        them; sums in FP64 here;
 *     2  BF16x3: each of those values v carried as hi + lo with
 *        hi = bf16(v), lo = bf16(v - hi) (the float difference is exact);
 *        a product a b is ahi bhi + ahi blo + alo bhi (lo lo dropped); the
 *        hidden sum is rounded to float before its split, as the GPU's FP32
 *        accumulator is.
 *   Odd part: f_odd(x) = (f(x) - f(-x)) / 2, evaluated literally; for a
 *         bias-free ReLU network it equals W2 W1 x / 2 (relu(a) - relu(-a)
 *         = a), a linear map.
 *   Backward (loss gradients): in modes 1 and 2 the backward products use
 *         bf16 copies (hi parts) of x, W2 and the hidden activations.
 *   Loss: L = sum over batch and outputs of (y - t)^2 / (B D).
 *   Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *         w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), in float.
 *   Preconditioner: u = Z (D^-1 r); per element rms_e = sqrt(mean u_e^2);
 *         y_e = rms_e MLP(u_e / rms_e) (0 where rms_e = 0), MLP = f or f_odd;
 *         z = D^-1 r + corr, corr_g = y_e at the element-interior node g of
 *         element e (1 <= i,j,k <= N-1; one element per interior node), 0 at
 *         every other node: the training targets (the element-interior
 *         error) vanish there, so those outputs are not used.
 *   FPCG: alpha = r.z / p.Ap; x += alpha p; r -= alpha Ap;
 *         z' = M(r); if r.z' <= 0 or not finite, z' = D^-1 r;
 *         beta = r.(z' - z) / (r_old.z_old); p = z' + beta p.
 *
 * Parity pinned by tests/test_oracle_pins.py (finite differences, positive
 * homogeneity, the odd part against W2 W1 x / 2, the BF16x3 error bound,
 * FPCG with W2 = 0 against Jacobi-PCG).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* bfloat16 round to nearest even of a float value (NaN kept quiet). */
static float bf16_round(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) { /* inf or nan */
    if (u & 0x007fffffu) u |= 0x00400000u;
    u &= 0xffff0000u;
  } else {
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
  }
  memcpy(&f, &u, 4);
  return f;
}

void bso_bf16_round(int64_t n, const float *in, float *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = bf16_round(in[i]);
}

static double rnd(double v, int bf16) { return bf16 ? (double)bf16_round((float)v) : v; }

/* a b in precision mode prec (a, b already float values in modes 1 and 2) */
static double prod(double a, double b, int prec) {
  if (prec == 0) return a * b;
  if (prec == 1) return rnd(a, 1) * rnd(b, 1);
  const float af = (float)a, bf = (float)b;
  const float ah = bf16_round(af), bh = bf16_round(bf);
  const double al = bf16_round(af - ah), bl = bf16_round(bf - bh);
  return (double)ah * bh + (double)ah * bl + al * (double)bh;
}

/* the hidden value as the next layer sees it (before its product rounding) */
static double hidden_val(double s, int prec) {
  if (prec == 0) return s;
  return prec == 1 ? rnd((float)s, 1) : (double)(float)s;
}

/* one row: y = f(x) (odd = 0) or f_odd(x) = (f(x) - f(-x)) / 2 (odd = 1);
 * h (H values) receives the hidden activations of f(x). */
static void forward_row(int D, int H, const float *W1, const float *W2, const float *x,
                        double *y, double *h, double *h2, int prec, int odd) {
  for (int pass = 0; pass < 1 + odd; ++pass) {
    const double sgn = pass ? -1.0 : 1.0;
    double *hh = pass ? h2 : h;
    for (int j = 0; j < H; ++j) {
      double s = 0.0;
      for (int i = 0; i < D; ++i) s += prod(W1[j * D + i], sgn * x[i], prec);
      hh[j] = hidden_val(s > 0.0 ? s : 0.0, prec);
    }
  }
  for (int i = 0; i < D; ++i) {
    double s = 0.0;
    for (int j = 0; j < H; ++j) s += prod(W2[i * H + j], h[j], prec);
    if (odd) {
      double s2 = 0.0;
      for (int j = 0; j < H; ++j) s2 += prod(W2[i * H + j], h2[j], prec);
      s = (s - s2) / 2.0;
    }
    y[i] = s;
  }
}

/* y[B x D] = f(x) or f_odd(x) per row; hid (optional, B x H) receives the
 * hidden activations of f(x) as used. */
void bso_mlp_forward(int64_t B, int D, int H, const float *W1, const float *W2,
                     const float *X, double *Y, double *hid, int prec, int odd) {
  double *h = malloc(sizeof(double) * 2 * H);
  if (!h) return;
  for (int64_t b = 0; b < B; ++b) {
    forward_row(D, H, W1, W2, X + b * D, Y + b * D, h, h + H, prec, odd);
    if (hid)
      for (int j = 0; j < H; ++j) hid[b * H + j] = h[j];
  }
  free(h);
}

/* MSE loss and gradients dL/dW1 (H x D), dL/dW2 (D x H). */
double bso_mlp_loss_grad(int64_t B, int D, int H, const float *W1, const float *W2,
                         const float *X, const float *T, double *gW1, double *gW2,
                         int prec) {
  const int bf16 = prec != 0;
  double *y = malloc(sizeof(double) * D), *h = malloc(sizeof(double) * H);
  double *dy = malloc(sizeof(double) * D), *dh = malloc(sizeof(double) * H);
  if (!y || !h || !dy || !dh) { free(y); free(h); free(dy); free(dh); return NAN; }
  for (int64_t k = 0; k < (int64_t)H * D; ++k) gW1[k] = 0.0;
  for (int64_t k = 0; k < (int64_t)D * H; ++k) gW2[k] = 0.0;
  double loss = 0.0;
  const double scale = 2.0 / ((double)B * D);
  for (int64_t b = 0; b < B; ++b) {
    const float *x = X + b * D;
    bso_mlp_forward(1, D, H, W1, W2, x, y, h, prec, 0);
    for (int i = 0; i < D; ++i) {
      const double e = y[i] - T[b * D + i];
      loss += e * e;
      dy[i] = scale * e;
    }
    for (int j = 0; j < H; ++j) h[j] = rnd(h[j], bf16);
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < H; ++j) gW2[i * H + j] += dy[i] * h[j];
    for (int j = 0; j < H; ++j) {
      double s = 0.0;
      for (int i = 0; i < D; ++i) s += rnd(W2[i * H + j], bf16) * dy[i];
      dh[j] = h[j] > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < H; ++j)
      for (int i = 0; i < D; ++i) gW1[j * D + i] += dh[j] * rnd(x[i], bf16);
  }
  free(y); free(h); free(dy); free(dh);
  return loss / ((double)B * D);
}

/* One Adam step on float weights w (n), step number t >= 1. */
void bso_adam(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1,
              float b2, float eps, int t) {
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0f - b1) * g[i];
    v[i] = b2 * v[i] + (1.0f - b2) * g[i] * g[i];
    const float mh = m[i] / c1, vh = v[i] / c2;
    w[i] = w[i] - lr * mh / (sqrtf(vh) + eps);
  }
}

/* ------------------------------------------------------------------------ */
/* Learned preconditioner and flexible PCG, on the operator of bs_oracle.c. */
/* ------------------------------------------------------------------------ */
int bso_apply_A(int E, int N, double h, double lambda, const double *coef,
                const int32_t *ids, int64_t NG, const double *p, double *Ap);
int bso_diag_A(int E, int N, double h, double lambda, const double *coef,
               const int32_t *ids, int64_t NG, double *diag);

/* z = D^-1 r + v^-1 Z^T (rms MLP(Z D^-1 r / rms)); W2 == NULL: z = D^-1 r. */
static void precond(int E, int N, const int32_t *ids, int64_t NG, const double *dg,
                    const float *W1, const float *W2, int H, int prec, int odd,
                    const double *r, double *z) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  for (int64_t g = 0; g < NG; ++g) z[g] = r[g] / dg[g];
  if (!W2) return;
  float *x = malloc(sizeof(float) * Np);
  double *y = malloc(sizeof(double) * Np), *corr = calloc((size_t)NG, sizeof(double));
  if (!x || !y || !corr) { free(x); free(y); free(corr); return; }
  for (int e = 0; e < E; ++e) {
    const int32_t *id = ids + (int64_t)e * Np;
    double ss = 0.0;
    for (int l = 0; l < Np; ++l) {
      const double u = id[l] >= 0 ? z[id[l]] : 0.0;
      ss += u * u;
    }
    const double rms = sqrt(ss / Np);
    if (!(rms > 0.0)) continue;
    for (int l = 0; l < Np; ++l) x[l] = (float)((id[l] >= 0 ? z[id[l]] : 0.0) / rms);
    bso_mlp_forward(1, Np, H, W1, W2, x, y, NULL, prec, odd);
    /* element-interior outputs only; each interior node has one element */
    for (int k = 1; k < N; ++k)
      for (int j = 1; j < N; ++j)
        for (int i = 1; i < N; ++i) {
          const int l = i + Nq * (j + Nq * k);
          if (id[l] >= 0) corr[id[l]] += rms * y[l];
        }
  }
  for (int64_t g = 0; g < NG; ++g) z[g] += corr[g];
  free(x); free(y); free(corr);
}

static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Flexible PCG; returns iterations (or -1 breakdown, -2 alloc); *fallbacks
 * counts iterations whose correction was rejected.
 *
 * The Jacobi judge (period > 0): after every `period`-th iteration the
 * residual is compared with the last one that marked progress; when r.r has
 * dropped to a quarter of it (the residual norm halved) this iterate marks
 * progress, otherwise once `stall` iterations have passed since the last
 * progress the learned correction is dropped for good and the iteration
 * restarts from the current x with the Jacobi preconditioner: z = D^-1 r,
 * p = z.  *switched_at receives that iteration (0: never). */
int bso_fpcg_judged(int E, int N, double h, double lambda, const double *coef,
                    const int32_t *ids, int64_t NG, const float *W1, const float *W2, int H,
                    int prec, int odd, const double *b, double *x, double tol, int maxit,
                    int period, int stall, double *hist_rr, int *fallbacks, int *switched_at) {
  double *buf = malloc(sizeof(double) * 6 * NG);
  if (!buf) return -2;
  double *r = buf, *p = r + NG, *Ap = p + NG, *z = Ap + NG, *zn = z + NG, *dg = zn + NG;
  bso_diag_A(E, N, h, lambda, coef, ids, NG, dg);
  for (int64_t g = 0; g < NG; ++g) x[g] = 0.0;
  for (int64_t g = 0; g < NG; ++g) r[g] = b[g];
  int fb = 0;
  precond(E, N, ids, NG, dg, W1, W2, H, prec, odd, r, z);
  double rz = dot(NG, r, z);
  if (!(rz > 0.0) || !isfinite(rz)) {
    for (int64_t g = 0; g < NG; ++g) z[g] = r[g] / dg[g];
    rz = dot(NG, r, z);
    ++fb;
  }
  for (int64_t g = 0; g < NG; ++g) p[g] = z[g];
  double rr = dot(NG, r, r);
  const double eps = tol * tol * dot(NG, b, b);
  if (hist_rr) hist_rr[0] = rr;
  int j = 0;
  double progress_rr = INFINITY;
  int progress_it = 0;
  if (switched_at) *switched_at = 0;
  while (j < maxit && rr > eps) {
    bso_apply_A(E, N, h, lambda, coef, ids, NG, p, Ap);
    const double pAp = dot(NG, p, Ap);
    if (!(pAp > 0.0) || !isfinite(pAp)) { free(buf); return -1; }
    const double alpha = rz / pAp;
    for (int64_t g = 0; g < NG; ++g) {
      x[g] = x[g] + alpha * p[g];
      r[g] = r[g] - alpha * Ap[g];
    }
    rr = dot(NG, r, r);
    ++j;
    if (hist_rr) hist_rr[j] = rr;
    if (rr <= eps) break;
    if (period > 0 && W2 && j % period == 0) {
      if (rr <= 0.25 * progress_rr) {
        progress_rr = rr;
        progress_it = j;
      } else if (j - progress_it >= stall) {
        W1 = NULL;  /* Jacobi from here on */
        W2 = NULL;
        if (switched_at) *switched_at = j;
        for (int64_t g = 0; g < NG; ++g) {
          z[g] = r[g] / dg[g];
          p[g] = z[g];
        }
        rz = dot(NG, r, z);
        continue;
      }
    }
    precond(E, N, ids, NG, dg, W1, W2, H, prec, odd, r, zn);
    double rzn = dot(NG, r, zn);
    if (!(rzn > 0.0) || !isfinite(rzn)) {
      for (int64_t g = 0; g < NG; ++g) zn[g] = r[g] / dg[g];
      rzn = dot(NG, r, zn);
      ++fb;
    }
    const double beta = (rzn - dot(NG, r, z)) / rz;
    for (int64_t g = 0; g < NG; ++g) {
      p[g] = zn[g] + beta * p[g];
      z[g] = zn[g];
    }
    rz = rzn;
  }
  if (fallbacks) *fallbacks = fb;
  free(buf);
  return j;
}

int bso_fpcg(int E, int N, double h, double lambda, const double *coef, const int32_t *ids,
             int64_t NG, const float *W1, const float *W2, int H, int prec, int odd,
             const double *b, double *x, double tol, int maxit, double *hist_rr,
             int *fallbacks) {
  return bso_fpcg_judged(E, N, h, lambda, coef, ids, NG, W1, W2, H, prec, odd, b, x, tol, maxit,
                         0, 0, hist_rr, fallbacks, NULL);
}
