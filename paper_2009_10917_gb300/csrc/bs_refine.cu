// bs_refine.cu -- CG with FP32 vectors inside an FP64 iterative-refinement
// loop (Algorithm 1 as the inner solver).
//
// Outer, in FP64 (the only FP64 steps on the GPU):
//   r = b - A x,  stop when ||r|| <= tol ||b||,  x = x + d.
// Inner, Algorithm 1 on A d = r with every vector and the operator in FP32:
// the same four kernels per iteration as the FP64 solver (fused scatter +
// element operator, gather with p.Ap, fused update with r.r, AXPY), their
// reductions carried as float pairs and combined in double, alpha and beta
// formed in double and rounded to float for the updates.  Each inner solve
// stops at ||r_d|| <= inner_tol ||r||.  Halving the bytes of every vector and
// moving the element operator from GB300's narrow FP64 pipe to the FP32
// pipes is what makes this faster than the FP64 solve at equal accuracy.
// Every inner solve starts afresh (d_0 = 0, p = r): keeping the search
// direction across a residual replacement was tried and stalled on
// ill-conditioned cases without saving iterations where it converged.
#include <chrono>
#include <cmath>
#include <cstring>

#include "bs_op_ff.cuh"

namespace bs {

// r = b - Ax (FP64), rf = (float) r, total = r.r; one pass.
__global__ void __launch_bounds__(kReduceBlock)
    k_residual(int64_t n, const double *__restrict__ b, const double *__restrict__ Ax,
               double *__restrict__ r, float *__restrict__ rf, double *partials,
               unsigned int *counter, double *out) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t i = tid; i < n; i += nth) {
    const double ri = b[i] - Ax[i];
    r[i] = ri;
    rf[i] = (float)ri;
    acc = fma(ri, ri, acc);
  }
  const double part = block_sum<kReduceBlock>(acc);
  double total;
  if (grid_combine<kReduceBlock>(part, partials, counter, &total) && threadIdx.x == 0)
    *out = total;
}

// x = x + (double) d
__global__ void k_add_f32(int64_t n, const float *__restrict__ d, double *__restrict__ x) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += nth) x[i] = x[i] + (double)d[i];
}

struct EpInitInner {  // inner r.r: the inner solve's b.b, its r_0.r_0 and stop rule
  CgState *st;
  double tol2;
  int maxit;
  __device__ __forceinline__ void operator()(double s) const {
    st->bb = s;
    st->rr = s;
    st->eps = tol2 * s;
    st->iter = 0;
    st->maxit = maxit;
    st->fixed = 0;
    st->hist = nullptr;
    st->done = !isfinite(s) ? 2 : ((s <= st->eps) ? 1 : (maxit <= 0 ? 3 : 0));
  }
};

struct EpAlphaF {  // pAp -> alpha (double, and rounded to float)
  CgState *st;
  __device__ __forceinline__ void operator()(double s) const {
    st->pAp = s;
    if (!(s > 0.0) || !isfinite(s)) {
      st->done = 2;
      return;
    }
    const double a = st->rr / s;
    st->alpha = a;
    st->alpha_f = (float)a;
  }
};

struct EpBetaF {  // rr' -> beta = rr'/rr, stop rule
  CgState *st;
  __device__ __forceinline__ void operator()(double s) const {
    const double beta = s / st->rr;
    const int j = st->iter;
    st->beta = beta;
    st->beta_f = (float)beta;
    st->rr = s;
    st->iter = j + 1;
    if (!isfinite(s) || !isfinite(beta))
      st->done = 2;
    else if (s <= st->eps)
      st->done = 1;
    else if (j + 1 >= st->maxit)
      st->done = 3;
  }
};

struct F32Vecs {
  float *r, *p, *Ap, *d;
};

static int ensure_f32(bs_problem *P) {
  if (P->d_f32) return BS_OK;
  const size_t n = (size_t)P->map->NG + 8;
  BS_CUDA_TRY(cudaMalloc(&P->d_f32, sizeof(float) * 4 * n));
  return BS_OK;
}

static F32Vecs f32vecs(const bs_problem *P) {
  const size_t n = (size_t)P->map->NG + 8;  // keeps each vector 16-byte aligned
  return F32Vecs{P->d_f32, P->d_f32 + n, P->d_f32 + 2 * n, P->d_f32 + 3 * n};
}

// One inner FP32 CG iteration (four launches).
static int f32_iteration(const bs_problem *P, cudaStream_t s) {
  const bs_map *m = P->map;
  F32Vecs v = f32vecs(P);
  CgState *st = P->d_state;
  float *ApL = reinterpret_cast<float *>(P->d_ApL);
  const float g = (float)(0.5 * P->h);
  const float mlam = (float)(P->lambda * 0.125 * P->h * P->h * P->h);
  int rc = apply_A_global<float, true, EpAlphaF>(P, false, P->d_tabf, v.p, v.Ap, ApL, g, mlam,
                                                  EpAlphaF{st}, st, s);
  if (rc) return rc;
  rc = launch_cg_update<float, EpBetaF>(m->NG, Scalar<float>{0.f, &st->alpha_f}, v.p, v.Ap, v.d,
                                        v.r, P->d_partials, P->d_counter, EpBetaF{st}, st, s);
  if (rc) return rc;
  return launch_axpy<float>(m->NG, Scalar<float>{1.f, nullptr}, v.r,
                            Scalar<float>{0.f, &st->beta_f}, v.p, st, s);
}

static int capture_f32(bs_problem *P, int chunk) {
  const void *key[4] = {nullptr, (const void *)(intptr_t)(2 | (g_op_fusion ? 4 : 0) |
                                                    (g_op_evenodd ? 16 : 0)),
                        (const void *)(intptr_t)chunk,
                        (const void *)P->map};
  if (P->graph && memcmp(key, P->graph_key, sizeof(key)) == 0) return BS_OK;
  if (P->graph) {
    cudaGraphExecDestroy(P->graph);
    P->graph = nullptr;
  }
  cudaStream_t cs = P->cap_stream;
  BS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int rc = BS_OK;
  for (int c = 0; c < chunk && rc == BS_OK; ++c) rc = f32_iteration(P, cs);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (rc != BS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(BS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&P->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    P->graph = nullptr;
    return fail(BS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  memcpy(P->graph_key, key, sizeof(key));
  return BS_OK;
}

}  // namespace bs

using namespace bs;

extern "C" int bs_cg_solve_refined_f32(const bs_problem *Pc, const double *b, double *x,
                                       double tol, int32_t maxit, double inner_tol,
                                       int32_t outer_maxit, int32_t flags, bs_cg_info *info,
                                       void *stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (info) memset(info, 0, sizeof(*info));
  BS_ARG(Pc != nullptr, "bs_cg_solve_refined_f32: problem is NULL");
  bs_problem *P = const_cast<bs_problem *>(Pc);
  int dev = -1;
  BS_CUDA_TRY(cudaGetDevice(&dev));
  BS_ARG(dev == P->device, "bs_cg_solve_refined_f32: problem belongs to device %d", P->device);
  BS_ARG(maxit >= 0 && outer_maxit >= 0, "bs_cg_solve_refined_f32: negative limit");
  BS_ARG(!P->d_geo, "bs_cg_solve_refined_f32: not available with geometric factors");
  BS_ARG(tol >= 0.0 && std::isfinite(tol), "bs_cg_solve_refined_f32: bad tol");
  BS_ARG(inner_tol > 0.0 && inner_tol < 1.0, "bs_cg_solve_refined_f32: inner_tol in (0, 1)");
  const bs_map *m = P->map;
  const int64_t NG = m->NG;
  BS_ARG(NG == 0 || (b && x), "bs_cg_solve_refined_f32: NULL vector");
  int rc = ensure_f32(P);
  if (rc) return rc;
  cudaStream_t s = as_stream(stream);
  const bool graph = flags & BS_CG_GRAPH;
  const int64_t sv = NG + 2;
  double *r64 = P->d_vec, *Ax = P->d_vec + 2 * sv, *scal = P->d_vec + 5 * sv;  // scal[0..1]
  F32Vecs v = f32vecs(P);
  CgState *st = P->d_state;
  const double g = 0.5 * P->h, mlam = P->lambda * g * g * g;
  const int chunk = 8;
  int total = 0, outer = 0;
  double bb = 0.0, rr = 0.0;
  if (!(flags & BS_CG_X0)) BS_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * NG, s));
  rc = launch_dot<double, true, EpStore>(NG, b, b, P->d_partials, P->d_counter,
                                         EpStore{scal + 1}, nullptr, s);
  if (rc) return rc;
  BS_CUDA_TRY(cudaMemcpyAsync(&bb, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  const int grid = stream_grid(NG, 1, kReduceBlock, 6);
  for (;;) {
    // outer residual in FP64
    rc = apply_A_global<double, false, EpNone>(P, false, P->d_tab, x, Ax, P->d_ApL, g, mlam,
                                               EpNone{}, nullptr, s);
    if (rc) break;
    k_residual<<<grid, kReduceBlock, 0, s>>>(NG, b, Ax, r64, v.r, P->d_partials, P->d_counter,
                                             scal);
    BS_CUDA_TRY(cudaMemcpyAsync(&rr, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    BS_CUDA_TRY(cudaStreamSynchronize(s));
    if (!std::isfinite(rr)) {
      rc = fail(BS_ERR_BREAKDOWN, "bs_cg_solve_refined_f32: non-finite residual");
      break;
    }
    if (rr <= tol * tol * bb) break;
    if (outer >= outer_maxit || total >= maxit) {
      rc = fail(BS_ERR_NOT_CONVERGED, "bs_cg_solve_refined_f32: %d outer, %d inner iterations",
                outer, total);
      break;
    }
    // inner FP32 CG on A d = r, d_0 = 0
    BS_CUDA_TRY(cudaMemsetAsync(v.d, 0, sizeof(float) * NG, s));
    rc = launch_copy<float>(NG, v.r, v.p, s);
    if (!rc)
      rc = launch_dot<float, true, EpInitInner>(NG, v.r, v.r, P->d_partials, P->d_counter,
                                                EpInitInner{st, inner_tol * inner_tol,
                                                            maxit - total},
                                                nullptr, s);
    if (!rc && graph) rc = capture_f32(P, chunk);
    if (rc) break;
    for (;;) {
      if (graph) {
        BS_CUDA_TRY(cudaGraphLaunch(P->graph, s));
      } else {
        for (int c = 0; c < chunk && !rc; ++c) rc = f32_iteration(P, s);
        if (rc) break;
      }
      BS_CUDA_TRY(cudaMemcpyAsync(P->h_state, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
      BS_CUDA_TRY(cudaStreamSynchronize(s));
      if (P->h_state->done) break;
    }
    if (rc) break;
    total += P->h_state->iter;
    if (P->h_state->done == 2) {
      rc = fail(BS_ERR_BREAKDOWN, "bs_cg_solve_refined_f32: inner breakdown");
      break;
    }
    k_add_f32<<<grid, kReduceBlock, 0, s>>>(NG, v.d, x);
    BS_LAUNCH_CHECK();
    ++outer;
  }
  if (info) {
    info->iterations = total;
    info->outer = outer;
    info->rr = rr;
    info->bb = bb;
    info->rel_residual = bb > 0 ? std::sqrt(rr / bb) : std::sqrt(rr);
    info->status = rc;
    info->seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}
