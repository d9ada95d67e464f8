// bs_cg.cu -- Algorithm 1 (conjugate gradients) on A x = b, strung together
// from the BS kernels with every scalar kept on the device.
//
// One iteration is four launches, none of which waits for the host:
//   1. ApL = A_L (Z p)                 fused scatter + element operator
//   2. Ap = Z^T ApL, pAp = p.Ap        gather (BS6) with a fused dot;
//                                      its last block forms alpha = rr / pAp
//   3. x += alpha p, r -= alpha Ap,    fused CG update (BS5); its last block
//      rr' = r.r                       forms beta = rr'/rr and the stop flag
//   4. p = r + beta p                  AXPY (BS2), p = fma(1, r, beta p)
// Kernels return at once when the device stop flag is set, so a chunk of
// iterations can be enqueued -- or replayed as one CUDA graph -- and the host
// reads the flag back once per chunk.
#include <chrono>
#include <cmath>

#include "bs_op_ff.cuh"

namespace bs {

struct EpBB {  // b.b
  CgState *st;
  __device__ __forceinline__ void operator()(double s) const { st->bb = s; }
};

struct EpInit {  // r_0.r_0 and the stopping rule
  CgState *st;
  double tol2;
  int maxit, fixed;
  double *hist;
  __device__ __forceinline__ void operator()(double s) const {
    st->rr = s;
    st->eps = tol2 * st->bb;
    st->iter = 0;
    st->maxit = maxit;
    st->fixed = fixed;
    st->hist = hist;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->done = !isfinite(s) ? 2 : ((!fixed && s <= st->eps) ? 1 : (maxit <= 0 ? 3 : 0));
  }
};

struct EpAlpha {  // pAp -> alpha = rr / pAp (rz / pAp when preconditioned)
  CgState *st;
  int precond;
  __device__ __forceinline__ void operator()(double s) const {
    st->pAp = s;
    if (!(s > 0.0) || !isfinite(s)) {
      st->done = 2;
      return;
    }
    const double a = (precond ? st->rz : st->rr) / s;
    st->alpha = a;
    st->alpha_f = (float)a;
  }
};

__device__ __forceinline__ void cg_advance(CgState *st, double rr_new, double beta) {
  const int j = st->iter;
  if (st->hist) {
    st->hist[3 * j] = st->alpha;
    st->hist[3 * j + 1] = beta;
    st->hist[3 * j + 2] = rr_new;
  }
  st->beta = beta;
  st->beta_f = (float)beta;
  st->rr = rr_new;
  st->iter = j + 1;
  if (!isfinite(rr_new) || !isfinite(beta))
    st->done = 2;
  else if (!st->fixed && rr_new <= st->eps)
    st->done = 1;
  else if (j + 1 >= st->maxit)
    st->done = 3;
}

struct EpBeta {  // rr' -> beta = rr'/rr (Algorithm 1, step 10)
  CgState *st;
  __device__ __forceinline__ void operator()(double s) const {
    cg_advance(st, s, s / st->rr);
  }
};

// Jacobi-PCG update: x += alpha p; r -= alpha Ap; z = dinv r; sums r.r, r.z.
template <int U>
__global__ void __launch_bounds__(kReduceBlock)
    k_pcg_update(int64_t n, const double *__restrict__ p, const double *__restrict__ Ap,
                 const double *__restrict__ dinv, double *__restrict__ x,
                 double *__restrict__ r, double *__restrict__ z, double *partials,
                 unsigned int *counter, CgState *st, int init) {
  if (!init && cg_halted(st)) return;
  const double alpha = init ? 0.0 : st->alpha;
  const double nalpha = -alpha;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  double rr = 0.0, rz = 0.0;
  for (int64_t i = tid; i < n; i += nth) {
    double ri = r[i];
    if (!init) {
      x[i] = fma(alpha, p[i], x[i]);
      ri = fma(nalpha, Ap[i], ri);
      r[i] = ri;
    }
    const double zi = ri * dinv[i];
    z[i] = zi;
    rr = fma(ri, ri, rr);
    rz = fma(ri, zi, rz);
  }
  const double prr = block_sum<kReduceBlock>(rr);
  const double prz = block_sum<kReduceBlock>(rz);
  double trr, trz;
  if (grid_combine2<kReduceBlock>(prr, prz, partials, counter, &trr, &trz) &&
      threadIdx.x == 0) {
    if (init) {
      st->rr = trr;
      st->rz = trz;
      st->done = !(isfinite(trr) && isfinite(trz))
                     ? 2
                     : ((!st->fixed && trr <= st->eps) ? 1 : (st->maxit <= 0 ? 3 : 0));
    } else {
      const double beta = trz / st->rz;
      st->rz = trz;
      cg_advance(st, trr, beta);
    }
  }
}

// v[i] = s * v[i] (s a power of two: exact).
__global__ void k_scale(int64_t n, double s, double *__restrict__ v) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += nth) v[i] = s * v[i];
}

__global__ void k_reciprocal(int64_t n, const double *__restrict__ d, double *__restrict__ inv) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += nth) inv[i] = 1.0 / d[i];
}

__global__ void k_set_state(CgState *st, double tol2, int maxit, int fixed, double *hist) {
  st->eps = tol2 * st->bb;
  st->iter = 0;
  st->maxit = maxit;
  st->fixed = fixed;
  st->hist = hist;
  st->alpha = 0.0;
  st->beta = 0.0;
}

struct CgVecs {
  double *r, *p, *Ap, *z, *dinv;
};
static CgVecs vecs(const bs_problem *P) {
  const int64_t s = P->map->NG + 2;
  return CgVecs{P->d_vec, P->d_vec + s, P->d_vec + 2 * s, P->d_vec + 3 * s, P->d_vec + 4 * s};
}

static int pcg_update_launch(const bs_problem *P, double *x, int init, cudaStream_t s) {
  CgVecs v = vecs(P);
  auto kern = k_pcg_update<1>;
  int grid = stream_grid(P->map->NG, 2, kReduceBlock, blocks_per_sm(kern, kReduceBlock));
  if (grid > kMaxPartials / 2) grid = kMaxPartials / 2;
  kern<<<grid, kReduceBlock, 0, s>>>(P->map->NG, v.p, v.Ap, v.dinv, x, v.r, v.z, P->d_partials,
                                     P->d_counter, P->d_state, init);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// One CG iteration (four launches: the operator with p.Ap, the fused update
// with r.r, the direction).  ff: the float-float element operator.
static int cg_iteration(const bs_problem *P, double *x, bool precond, bool ff, cudaStream_t s) {
  const bs_map *m = P->map;
  CgVecs v = vecs(P);
  CgState *st = P->d_state;
  const double g = 0.5 * P->h, mlam = P->lambda * g * g * g;
  int rc = apply_A_global<double, true, EpAlpha>(P, ff, P->d_tab, v.p, v.Ap, P->d_ApL, g, mlam,
                                                 EpAlpha{st, precond ? 1 : 0}, st, s);
  if (rc) return rc;
  if (precond) {
    rc = pcg_update_launch(P, x, 0, s);
  } else {
    rc = launch_cg_update<double, EpBeta>(m->NG, Scalar<double>{0.0, &st->alpha}, v.p, v.Ap, x,
                                          v.r, P->d_partials, P->d_counter, EpBeta{st}, st, s);
  }
  if (rc) return rc;
  return launch_axpy<double>(m->NG, Scalar<double>{1.0, nullptr}, precond ? v.z : v.r,
                             Scalar<double>{0.0, &st->beta}, v.p, st, s);
}

static int capture_chunk(bs_problem *P, double *x, bool precond, bool ff, int chunk) {
  const void *key[4] = {x, (const void *)(intptr_t)((precond ? 1 : 0) | (ff ? 2 : 0) |
                                                     (g_op_fusion ? 4 : 0)),
                        (const void *)(intptr_t)chunk,
                        (const void *)P->map};
  if (P->graph && key[0] == P->graph_key[0] && key[1] == P->graph_key[1] &&
      key[2] == P->graph_key[2] && key[3] == P->graph_key[3])
    return BS_OK;
  if (P->graph) {
    cudaGraphExecDestroy(P->graph);
    P->graph = nullptr;
  }
  cudaStream_t cs = P->cap_stream;
  BS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int rc = BS_OK;
  for (int c = 0; c < chunk && rc == BS_OK; ++c) rc = cg_iteration(P, x, precond, ff, cs);
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
  for (int i = 0; i < 4; ++i) P->graph_key[i] = key[i];
  return BS_OK;
}

}  // namespace bs

using namespace bs;

extern "C" int bs_cg_solve(const bs_problem *Pc, const double *b, double *x, double tol,
                           int32_t maxit, int32_t flags, double *d_hist, bs_cg_info *info,
                           void *stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (info) memset(info, 0, sizeof(*info));
  BS_ARG(Pc != nullptr, "bs_cg_solve: problem is NULL");
  bs_problem *P = const_cast<bs_problem *>(Pc);
  int dev = -1;
  BS_CUDA_TRY(cudaGetDevice(&dev));
  BS_ARG(dev == P->device, "bs_cg_solve: problem belongs to device %d", P->device);
  BS_ARG(maxit >= 0, "bs_cg_solve: maxit < 0");
  BS_ARG(tol >= 0.0 && std::isfinite(tol), "bs_cg_solve: tol must be finite and >= 0");
  const bs_map *m = P->map;
  const int64_t NG = m->NG;
  BS_ARG(NG == 0 || (b && x), "bs_cg_solve: NULL vector");
  cudaStream_t s = as_stream(stream);
  const bool fixed = flags & BS_CG_FIXED_ITERS;
  const bool precond = flags & BS_CG_JACOBI;
  const bool ff = flags & BS_CG_FF_OPERATOR;
  double ff_scale = 1.0;  // power of two the FF solve runs scaled by
  CgVecs v = vecs(P);
  CgState *st = P->d_state;
  int rc = BS_OK;
#define BS_TRY(expr)              \
  do {                            \
    if ((rc = (expr)) != BS_OK) { \
      goto done;                  \
    }                             \
  } while (0)
  {
    if (!(flags & BS_CG_X0)) BS_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * NG, s));
    if (ff && NG > 0) {
      // The float-float operator counts inputs below 2^-102 as zero: solve
      // the system scaled by the power of two that brings b's RMS near 1
      // (exact both ways), with the scaled b in the spare vector.
      BS_TRY((launch_dot<double, true, EpBB>(NG, b, b, P->d_partials, P->d_counter, EpBB{st},
                                             nullptr, s)));
      BS_CUDA_TRY(cudaMemcpyAsync(P->h_state, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
      BS_CUDA_TRY(cudaStreamSynchronize(s));
      const double bb0 = P->h_state->bb;
      if (bb0 > 0.0 && std::isfinite(bb0)) {
        ff_scale = std::ldexp(1.0, -std::ilogb(std::sqrt(bb0 / (double)NG)));
        double *bs_ = P->d_vec + 5 * (NG + 2);
        BS_TRY(launch_copy<double>(NG, b, bs_, s));
        const int grid = stream_grid(NG, 1, kStreamBlock, 8);
        k_scale<<<grid, kStreamBlock, 0, s>>>(NG, ff_scale, bs_);
        if (flags & BS_CG_X0) k_scale<<<grid, kStreamBlock, 0, s>>>(NG, ff_scale, x);
        BS_CUDA_TRY(cudaGetLastError());
        b = bs_;
      }
    }
    BS_TRY((launch_dot<double, true, EpBB>(NG, b, b, P->d_partials, P->d_counter, EpBB{st},
                                           nullptr, s)));
    // r_0 = b - A x_0
    BS_TRY(launch_copy<double>(NG, b, v.r, s));
    if (flags & BS_CG_X0) {
      BS_TRY(ff ? bs_apply_A_ff(P, x, v.Ap, stream) : bs_apply_A(P, x, v.Ap, stream));
      BS_TRY(launch_axpy<double>(NG, Scalar<double>{-1.0, nullptr}, v.Ap,
                                 Scalar<double>{1.0, nullptr}, v.r, nullptr, s));
    }
    if (precond) {
      BS_TRY(bs_diag_A(P, v.Ap, stream));
      const int grid = stream_grid(NG, 1, kStreamBlock, 8);
      k_reciprocal<<<grid, kStreamBlock, 0, s>>>(NG, v.Ap, v.dinv);
      k_set_state<<<1, 1, 0, s>>>(st, tol * tol, maxit, fixed ? 1 : 0, d_hist);
      BS_TRY(pcg_update_launch(P, x, 1, s));  // z = dinv r, rr, rz, stop flag
      BS_TRY(launch_copy<double>(NG, v.z, v.p, s));
    } else {
      BS_TRY(launch_copy<double>(NG, v.r, v.p, s));
      BS_TRY((launch_dot<double, true, EpInit>(
          NG, v.r, v.r, P->d_partials, P->d_counter,
          EpInit{st, tol * tol, maxit, fixed ? 1 : 0, d_hist}, nullptr, s)));
    }
    const bool graph = flags & BS_CG_GRAPH;
    const int chunk = maxit < 8 ? (maxit < 1 ? 1 : maxit) : 8;
    int launched = 0;
    if (graph && maxit > 0) BS_TRY(capture_chunk(P, x, precond, ff, chunk));
    while (launched < maxit) {
      if (graph) {
        BS_CUDA_TRY(cudaGraphLaunch(P->graph, s));
      } else {
        for (int c = 0; c < chunk; ++c) BS_TRY(cg_iteration(P, x, precond, ff, s));
      }
      launched += chunk;
      BS_CUDA_TRY(cudaMemcpyAsync(P->h_state, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
      BS_CUDA_TRY(cudaStreamSynchronize(s));
      if (P->h_state->done) break;
    }
    BS_CUDA_TRY(cudaMemcpyAsync(P->h_state, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    BS_CUDA_TRY(cudaStreamSynchronize(s));
    const CgState &h = *P->h_state;
    if (h.done == 2)
      rc = fail(BS_ERR_BREAKDOWN,
                "bs_cg_solve: breakdown at iteration %d (p.Ap = %g, r.r = %g)", h.iter, h.pAp,
                h.rr);
    else if (!fixed && !(h.rr <= h.eps))
      rc = fail(BS_ERR_NOT_CONVERGED, "bs_cg_solve: %d iterations, rel. residual %g", h.iter,
                h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0);
    if (info) {
      info->iterations = h.iter;
      info->rr = h.rr / (ff_scale * ff_scale);
      info->bb = h.bb / (ff_scale * ff_scale);
      info->rel_residual = h.bb > 0 ? std::sqrt(h.rr / h.bb) : std::sqrt(h.rr);
    }
    if (ff_scale != 1.0) {  // back to the unscaled solution (exact)
      k_scale<<<stream_grid(NG, 1, kStreamBlock, 8), kStreamBlock, 0, s>>>(NG, 1.0 / ff_scale, x);
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        rc = fail(BS_ERR_CUDA, "bs_cg_solve: unscaling the solution failed");
    }
  }
done:
#undef BS_TRY
  if (info) {
    info->status = rc;
    info->seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}
