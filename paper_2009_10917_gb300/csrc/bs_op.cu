// bs_op.cu -- GLL tables (host), problem objects and the C ABI of the
// operator A = Z^T (c S_L + lambda M_L) Z (eqs. global_system,
// assembled_stiff, assembled_mass).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <thread>
#include <vector>

#include "bs_op_ff.cuh"

namespace bs {

int g_op_fusion = 0;
int g_op_evenodd = 1;

// GLL nodes on [-1, 1] (Sec. 2, eq. basis): the N+1 zeros of (1 - x^2) P_N'(x).
// Newton on the Legendre-Vandermonde recurrence
//   x <- x - (x P_N(x) - P_{N-1}(x)) / ((N + 1) P_N(x)),
// started from the Chebyshev-Lobatto points cos(pi i / N), converges to all
// N+1 nodes, endpoints included.  Weights 2 / (N (N+1) P_N(x_i)^2).  The
// derivative matrix D[a][i] = l_i'(x_a) comes from barycentric weights
// b_j = 1 / prod_{k != j} (x_j - x_k):
//   D[a][i] = (b_i / b_a) / (x_a - x_i)  (a != i),  D[a][a] = -sum_{i != a} D[a][i].
static void gll_tables(int N, double *x, double *w, double *D) {
  const int Nq = N + 1;
  const double pi = 3.141592653589793238462643383279502884;
  std::vector<double> P((size_t)Nq * Nq);
  for (int i = 0; i <= N; ++i) x[i] = std::cos(pi * (N - i) / N);  // ascending
  for (int it = 0; it < 200; ++it) {
    double change = 0.0;
    for (int i = 0; i <= N; ++i) {
      double p0 = 1.0, p1 = x[i];
      for (int k = 2; k <= N; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x[i] * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_N, p0 = P_{N-1}
      const double dx = (x[i] * p1 - p0) / (Nq * p1);
      x[i] -= dx;
      change = std::fmax(change, std::fabs(dx));
    }
    if (change < 1e-16) break;
  }
  for (int i = 0; i <= N / 2; ++i) {  // exact symmetry
    const double s = 0.5 * (x[N - i] - x[i]);
    x[i] = -s;
    x[N - i] = s;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int i = 0; i <= N; ++i) {
    double p0 = 1.0, p1 = x[i];
    for (int k = 2; k <= N; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x[i] * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    w[i] = 2.0 / (N * (N + 1.0) * p1 * p1);
  }
  std::vector<double> b(Nq, 1.0);
  for (int j = 0; j <= N; ++j) {
    for (int k = 0; k <= N; ++k)
      if (k != j) b[j] *= (x[j] - x[k]);
    b[j] = 1.0 / b[j];
  }
  for (int a = 0; a <= N; ++a) {
    double diag = 0.0;
    for (int i = 0; i <= N; ++i) {
      if (i == a) continue;
      const double v = (b[i] / b[a]) / (x[a] - x[i]);
      D[a * Nq + i] = v;
      diag -= v;
    }
    D[a * Nq + a] = diag;
  }
}

// K = D^T W D, the 1-D stiffness on [-1, 1].
static void stiffness_1d(int N, const double *w, const double *D, double *K) {
  const int Nq = N + 1;
  for (int i = 0; i < Nq; ++i)
    for (int m = 0; m < Nq; ++m) {
      double s = 0.0;
      for (int a = 0; a < Nq; ++a) s = std::fma(D[a * Nq + i] * w[a], D[a * Nq + m], s);
      K[i * Nq + m] = s;
    }
}

// diag(A_L) per local node: c_e (h/2) (K_ii w_j w_k + w_i K_jj w_k + w_i w_j K_kk)
// + lambda (h/2)^3 w_i w_j w_k.
template <typename T>
__global__ void k_diag_local(int64_t NL, int Nq, const OpTab<T> *__restrict__ tab,
                             const double *__restrict__ coef, T g, T mlam,
                             T *__restrict__ out) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t Np = (int64_t)Nq * Nq * Nq;
  for (int64_t l = tid; l < NL; l += nth) {
    const int64_t e = l / Np;
    const int r = (int)(l - e * Np);
    const int i = r % Nq, j = (r / Nq) % Nq, k = r / (Nq * Nq);
    const T wi = tab->w[i], wj = tab->w[j], wk = tab->w[k];
    T s = tab->K[i * Nq + i] * wj * wk;
    s = s + wi * tab->K[j * Nq + j] * wk;
    s = s + wi * wj * tab->K[k * Nq + k];
    const T c = coef ? T(coef[e]) : T(1);
    out[l] = fmaT(c * g, s, mlam * (wi * wj * wk));
  }
}

static int check_prob(const bs_problem *p, const char *fn) {
  if (!p) return fail(BS_ERR_ARG, "%s: problem is NULL", fn);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
    return fail(BS_ERR_ARG, "%s: problem belongs to device %d, current is %d", fn, p->device,
                dev);
  return BS_OK;
}

static void free_problem(bs_problem *p) {
  if (!p) return;
  if (p->graph) cudaGraphExecDestroy(p->graph);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->d_coef);
  cudaFree(p->d_geo);
  cudaFree(p->d_tab);
  cudaFree(p->d_tabf);
  cudaFree(p->d_tabff);
  cudaFree(p->d_ApL);
  cudaFree(p->d_vec);
  cudaFree(p->d_state);
  cudaFree(p->d_partials);
  cudaFree(p->d_op_partials);
  cudaFree(p->d_f32);
  cudaFree(p->d_Lvec);
  cudaFree(p->d_owner);
  cudaFree(p->d_bj);
  if (p->h_state) cudaFreeHost(p->h_state);
  free(p);
}

// diag(A_L) per local node n = (i, j, k): the unit vector's quadratic form,
//   c_e [sum_m D_mi^2 G_rr(m,j,k) + sum_m D_mj^2 G_ss(i,m,k) + sum_m D_mk^2 G_tt(i,j,m)
//        + 2 (D_ii D_jj G_rs + D_ii D_kk G_rt + D_jj D_kk G_st)(n)] + lambda M_n
// (grad_r l_n is nonzero only on the three lines through n, and two of its
// components only at n itself).
static __global__ void k_diag_geo(int64_t NL, int Nq, const OpTab<double> *__restrict__ tab,
                           const double *__restrict__ coef, const double *__restrict__ geo,
                           double lambda, double *__restrict__ out) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int Nq2 = Nq * Nq, Np = Nq2 * Nq;
  const double *D = tab->D;
  for (int64_t l = tid; l < NL; l += nth) {
    const int64_t e = l / Np;
    const int n = (int)(l - e * Np);
    const int i = n % Nq, j = (n / Nq) % Nq, k = n / Nq2;
    const int64_t b = e * Np;
    double s = 0.0;
    for (int m = 0; m < Nq; ++m) {
      const double di = D[m * Nq + i], dj = D[m * Nq + j], dk = D[m * Nq + k];
      s = fma(di * di, geo[b + m + Nq * j + Nq2 * k], s);
      s = fma(dj * dj, geo[3 * NL + b + i + Nq * m + Nq2 * k], s);
      s = fma(dk * dk, geo[5 * NL + b + i + Nq * j + Nq2 * m], s);
    }
    const double dii = D[i * Nq + i], djj = D[j * Nq + j], dkk = D[k * Nq + k];
    s = fma(2.0 * dii * djj, geo[NL + l], s);
    s = fma(2.0 * dii * dkk, geo[2 * NL + l], s);
    s = fma(2.0 * djj * dkk, geo[4 * NL + l], s);
    out[l] = fma(coef ? coef[e] : 1.0, s, lambda * geo[6 * NL + l]);
  }
}

}  // namespace bs

using namespace bs;

extern "C" {

int bs_problem_create(const bs_map *map, double h, double lambda, const double *h_coef,
                      bs_problem **out) {
  BS_ARG(out != nullptr, "bs_problem_create: out is NULL");
  *out = nullptr;
  BS_ARG(map != nullptr, "bs_problem_create: map is NULL");
  BS_ARG(h > 0.0 && std::isfinite(h), "bs_problem_create: h must be positive");
  BS_ARG(lambda >= 0.0 && std::isfinite(lambda), "bs_problem_create: lambda must be >= 0");
  const int N = map->N, Nq = N + 1;
  BS_ARG(Nq <= kMaxNq, "bs_problem_create: degree %d unsupported", N);
  if (h_coef)
    for (int64_t e = 0; e < map->E; ++e)
      BS_ARG(h_coef[e] > 0.0 && std::isfinite(h_coef[e]),
             "bs_problem_create: coef[%lld] must be positive", (long long)e);
  bs_problem *p = (bs_problem *)calloc(1, sizeof(bs_problem));
  if (!p) return fail(BS_ERR_ALLOC, "bs_problem_create: host allocation");
  p->map = map;
  p->N = N;
  p->h = h;
  p->lambda = lambda;
  double x[kMaxNq], w[kMaxNq], D[kMaxNq * kMaxNq], K[kMaxNq * kMaxNq];
  gll_tables(N, x, w, D);
  stiffness_1d(N, w, D, K);
  OpTab<double> tab{};
  OpTab<float> tabf{};
  OpTabFF tabff{};
  // float pairs v = hi + lo (hi = v rounded to float, lo = the rest rounded)
  auto split = [](double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  if (Nq % 2 == 0) {  // even-odd halves of W^-1 K, centrosymmetrised
    const int hq = Nq / 2;
    auto kh = [&](int a, int m) {
      return 0.5 * (K[a * Nq + m] / w[a] + K[(Nq - 1 - a) * Nq + (Nq - 1 - m)] / w[Nq - 1 - a]);
    };
    for (int a = 0; a < hq; ++a)
      for (int m = 0; m < hq; ++m) {
        const double e = 0.5 * (kh(a, m) + kh(a, Nq - 1 - m));
        const double o = 0.5 * (kh(a, m) - kh(a, Nq - 1 - m));
        tab.Ee[a * hq + m] = e;
        tab.Eo[a * hq + m] = o;
        tabf.Ee[a * hq + m] = (float)e;
        tabf.Eo[a * hq + m] = (float)o;
        split(e, tabff.Eeh[a * hq + m], tabff.Eel[a * hq + m]);
        split(o, tabff.Eoh[a * hq + m], tabff.Eol[a * hq + m]);
      }
  }
  for (int i = 0; i < Nq; ++i) {
    tab.w[i] = w[i];
    tabf.w[i] = (float)w[i];
    split(w[i], tabff.wh[i], tabff.wl[i]);
    for (int m = 0; m < Nq; ++m) {
      tab.K[i * Nq + m] = K[i * Nq + m];
      tab.D[i * Nq + m] = D[i * Nq + m];
      tabf.D[i * Nq + m] = (float)D[i * Nq + m];
      split(D[i * Nq + m], tabff.Dh[i * Nq + m], tabff.Dl[i * Nq + m]);
      tabf.K[i * Nq + m] = (float)K[i * Nq + m];
      split(K[i * Nq + m], tabff.Kh[i * Nq + m], tabff.Kl[i * Nq + m]);
      split(w[i] * w[m], tabff.Wh[i * Nq + m], tabff.Wl[i * Nq + m]);
    }
  }
  const int64_t NL = map->NL, NG = map->NG;
  tab.ne = tabf.ne = tabff.ne = map->E;
  tab.ng = tabf.ng = tabff.ng = NG;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess && h_coef) e = cudaMalloc(&p->d_coef, sizeof(double) * (map->E + 1));
  if (e == cudaSuccess && h_coef)
    e = cudaMemcpy(p->d_coef, h_coef, sizeof(double) * map->E, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_tab, sizeof(tab));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_tabf, sizeof(tabf));
  if (e == cudaSuccess) e = cudaMemcpy(p->d_tab, &tab, sizeof(tab), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_tabf, &tabf, sizeof(tabf), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_tabff, sizeof(tabff));
  if (e == cudaSuccess) e = cudaMemcpy(p->d_tabff, &tabff, sizeof(tabff), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_ApL, sizeof(double) * (NL + 2));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_vec, sizeof(double) * 6 * (NG + 2));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_state, sizeof(CgState));
  if (e == cudaSuccess) e = cudaMemset(p->d_state, 0, sizeof(CgState));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_partials, sizeof(double) * kMaxPartials + 256);
  if (e == cudaSuccess) e = cudaMemset(p->d_partials, 0, sizeof(double) * kMaxPartials + 256);
  // one partial per element-kernel block: at most one block per element,
  // whichever kernel form (direct, even-odd) a later call selects
  if (e == cudaSuccess) e = cudaMalloc(&p->d_op_partials, sizeof(double) * (map->E + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_state, sizeof(CgState));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_problem(p);
    return fail(BS_ERR_CUDA, "bs_problem_create: %s", cudaGetErrorString(e));
  }
  p->d_counter = (unsigned int *)(p->d_partials + kMaxPartials);
  *out = p;
  return BS_OK;
}

int bs_problem_create_geo(const bs_map *map, double lambda, const double *h_coef,
                          const double *h_verts, bs_problem **out) {
  BS_ARG(out != nullptr, "bs_problem_create_geo: out is NULL");
  *out = nullptr;
  BS_ARG(map != nullptr, "bs_problem_create_geo: map is NULL");
  BS_ARG(map->N + 1 <= kGeoMaxNq, "bs_problem_create_geo: degree %d > %d", map->N,
         kGeoMaxNq - 1);
  BS_ARG(map->E == 0 || h_verts != nullptr, "bs_problem_create_geo: verts is NULL");
  const int N = map->N, Nq = N + 1, Np = Nq * Nq * Nq;
  const int64_t E = map->E, NL = map->NL;
  double x[kMaxNq], w[kMaxNq], D[kMaxNq * kMaxNq];
  gll_tables(N, x, w, D);
  // G = w det J J^-1 J^-T (upper triangle) and M = w det J at every node,
  // J = dx/dr of the trilinear map of the element's eight corners
  std::vector<double> fac((size_t)kGeoFactors * (size_t)NL);
  // elements split over host threads; bad[t] is the first degenerate
  // element thread t met (or -1)
  const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<int64_t> bad((size_t)nth, -1);
  auto work = [&](int t) {
  for (int64_t e = t; e < E; e += nth) {
    const double *X = h_verts + 24 * e;
    for (int n = 0; n < Np; ++n) {
      const int i = n % Nq, j = (n / Nq) % Nq, k = n / (Nq * Nq);
      const double r = x[i], s = x[j], t = x[k];
      double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      for (int v = 0; v < 8; ++v) {
        const double sx = (v & 1) ? 1.0 : -1.0, sy = (v & 2) ? 1.0 : -1.0,
                     sz = (v & 4) ? 1.0 : -1.0;
        const double dr = 0.125 * sx * (1.0 + sy * s) * (1.0 + sz * t);
        const double ds = 0.125 * (1.0 + sx * r) * sy * (1.0 + sz * t);
        const double dt = 0.125 * (1.0 + sx * r) * (1.0 + sy * s) * sz;
        for (int d = 0; d < 3; ++d) {
          J[d][0] += X[3 * v + d] * dr;
          J[d][1] += X[3 * v + d] * ds;
          J[d][2] += X[3 * v + d] * dt;
        }
      }
      // adjugate: C[p][d] = cofactor, J^-1 = C / det (rows: reference p)
      double C[3][3];
      C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      C[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
      C[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
      C[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
      C[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
      C[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      C[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
      C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      const double det = J[0][0] * C[0][0] + J[0][1] * C[1][0] + J[0][2] * C[2][0];
      if (!(det > 0.0) || !std::isfinite(det)) {
        if (bad[(size_t)t] < 0) bad[(size_t)t] = e;
        continue;
      }
      const double wq = w[i] * w[j] * w[k];
      // w det J (C/det)(C/det)^T = (w / det) C C^T
      const double sc = wq / det;
      auto cc = [&](int p, int q) {
        return C[p][0] * C[q][0] + C[p][1] * C[q][1] + C[p][2] * C[q][2];
      };
      const size_t l = (size_t)(e * Np + n);
      fac[0 * (size_t)NL + l] = sc * cc(0, 0);
      fac[1 * (size_t)NL + l] = sc * cc(0, 1);
      fac[2 * (size_t)NL + l] = sc * cc(0, 2);
      fac[3 * (size_t)NL + l] = sc * cc(1, 1);
      fac[4 * (size_t)NL + l] = sc * cc(1, 2);
      fac[5 * (size_t)NL + l] = sc * cc(2, 2);
      fac[6 * (size_t)NL + l] = wq * det;
    }
  }
  };
  {
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto &th : pool) th.join();
  }
  for (int64_t b : bad)
    if (b >= 0)
      return fail(BS_ERR_ARG, "bs_problem_create_geo: element %lld is inverted or degenerate",
                  (long long)b);
  bs_problem *p = nullptr;
  if (int rc = bs_problem_create(map, 1.0, lambda, h_coef, &p)) return rc;
  cudaError_t err = cudaMalloc(&p->d_geo, sizeof(double) * (fac.size() + 1));
  if (err == cudaSuccess && !fac.empty())
    err = cudaMemcpy(p->d_geo, fac.data(), sizeof(double) * fac.size(), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    free_problem(p);
    return fail(BS_ERR_CUDA, "bs_problem_create_geo: %s", cudaGetErrorString(err));
  }
  *out = p;
  return BS_OK;
}

int bs_problem_destroy(bs_problem *p) {
  free_problem(p);
  return BS_OK;
}

int bs_apply_local(const bs_problem *p, const double *uL, double *AuL, void *stream) {
  if (int rc = check_prob(p, "bs_apply_local")) return rc;
  if (p->map->NL == 0) return BS_OK;
  BS_ARG(uL && AuL, "bs_apply_local: NULL vector");
  const double g = 0.5 * p->h, mlam = p->lambda * g * g * g;
  if (p->d_geo)
    return launch_ax_geo<false>(p->N, p->map->E, p->map->NL, nullptr, nullptr, uL, AuL,
                                p->d_tab, p->d_coef, p->d_geo, p->lambda, nullptr,
                                as_stream(stream));
  return launch_ax_local<double, false>(p->N, p->map->E, nullptr, nullptr, uL, AuL, p->d_tab,
                                        p->d_coef, g, mlam, nullptr, as_stream(stream));
}

int bs_apply_A(const bs_problem *p, const double *x, double *Ax, void *stream) {
  if (int rc = check_prob(p, "bs_apply_A")) return rc;
  if (p->map->NG == 0) return BS_OK;
  BS_ARG(x && Ax, "bs_apply_A: NULL vector");
  const double g = 0.5 * p->h, mlam = p->lambda * g * g * g;
  return apply_A_global<double, false, EpNone>(p, false, p->d_tab, x, Ax, p->d_ApL, g, mlam,
                                               EpNone{}, nullptr, as_stream(stream));
}

int bs_apply_A_ff(const bs_problem *p, const double *x, double *Ax, void *stream) {
  if (int rc = check_prob(p, "bs_apply_A_ff")) return rc;
  if (p->map->NG == 0) return BS_OK;
  BS_ARG(x && Ax, "bs_apply_A_ff: NULL vector");
  const double g = 0.5 * p->h, mlam = p->lambda * g * g * g;
  return apply_A_global<double, false, EpNone>(p, true, p->d_tab, x, Ax, p->d_ApL, g, mlam,
                                               EpNone{}, nullptr, as_stream(stream));
}

int bs_diag_A(const bs_problem *p, double *d_diag, void *stream) {
  if (int rc = check_prob(p, "bs_diag_A")) return rc;
  if (p->map->NG == 0) return BS_OK;
  BS_ARG(d_diag != nullptr, "bs_diag_A: NULL output");
  const double g = 0.5 * p->h, mlam = p->lambda * g * g * g;
  cudaStream_t s = as_stream(stream);
  if (p->map->NL > 0) {
    const int grid = stream_grid(p->map->NL, 1, kStreamBlock, 8);
    if (p->d_geo)
      k_diag_geo<<<grid, kStreamBlock, 0, s>>>(p->map->NL, p->N + 1, p->d_tab, p->d_coef,
                                               p->d_geo, p->lambda, p->d_ApL);
    else
      k_diag_local<double><<<grid, kStreamBlock, 0, s>>>(p->map->NL, p->N + 1, p->d_tab,
                                                        p->d_coef, g, mlam, p->d_ApL);
    BS_LAUNCH_CHECK();
  }
  return launch_gather<double, false, EpNone>(p->map, p->d_ApL, d_diag, nullptr, nullptr,
                                              nullptr, EpNone{}, nullptr, s);
}

int bs_operator_mode(int32_t mode) {
  const int prev = (g_op_fusion ? BS_OP_FUSED : 0) | (g_op_evenodd ? 0 : BS_OP_DIRECT);
  if (mode >= 0) {
    g_op_fusion = (mode & BS_OP_FUSED) ? 1 : 0;
    g_op_evenodd = (mode & BS_OP_DIRECT) ? 0 : 1;
  }
  return prev;
}

}  // extern "C"
