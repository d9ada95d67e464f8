// bs_op.cu -- GLL tables (host), problem objects and the C ABI of the
// operator A = Z^T (c S_L + lambda M_L) Z (eqs. global_system,
// assembled_stiff, assembled_mass).
#include <cmath>
#include <cstdlib>
#include <cstring>
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
  if (p->h_state) cudaFreeHost(p->h_state);
  free(p);
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
      tabf.K[i * Nq + m] = (float)K[i * Nq + m];
      split(K[i * Nq + m], tabff.Kh[i * Nq + m], tabff.Kl[i * Nq + m]);
      split(w[i] * w[m], tabff.Wh[i * Nq + m], tabff.Wl[i * Nq + m]);
    }
  }
  const int64_t NL = map->NL, NG = map->NG;
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
  if (e == cudaSuccess)
    e = cudaMalloc(&p->d_op_partials, sizeof(double) * (ax_blocks(N, map->E) + 1));
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

int bs_problem_destroy(bs_problem *p) {
  free_problem(p);
  return BS_OK;
}

int bs_apply_local(const bs_problem *p, const double *uL, double *AuL, void *stream) {
  if (int rc = check_prob(p, "bs_apply_local")) return rc;
  if (p->map->NL == 0) return BS_OK;
  BS_ARG(uL && AuL, "bs_apply_local: NULL vector");
  const double g = 0.5 * p->h, mlam = p->lambda * g * g * g;
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
    k_diag_local<double><<<grid, kStreamBlock, 0, s>>>(p->map->NL, p->N + 1, p->d_tab, p->d_coef,
                                                      g, mlam, p->d_ApL);
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
