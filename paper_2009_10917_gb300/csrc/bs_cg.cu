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
//
// Scattered storage (BS_CG_SCATTERED; Sec. 3 sets it against global
// storage): Z applied to both sides of A x = b, so every vector is kept as
// v_L = Z v_G (N_L entries, masked ones zero) and A p = Z Z^T A_L p_L.  An
// inner product of two such vectors equals the global one when it sums one
// copy of each node -- the lowest local index, marked in an owner mask -- so
// the iterates are those of global CG up to summation order.  Five launches:
//   1. w_L = A_L p_L                   element kernel on contiguous data
//   2. Ap_G = Z^T w_L                  gather (BS6)
//   3. Ap_L = Z Ap_G, pAp over owners  scatter (BS7) with a fused dot; alpha
//   4. x_L, r_L update, r.r over owners
//   5. p_L = r_L + beta p_L
#include <chrono>
#include <cmath>

#include "bs_bj.cuh"
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
                 unsigned int *counter, CgState *st, int init, int defer) {
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
    } else if (defer) {  // block Jacobi completes z and r.z, then advances
      st->rr_next = trr;
      st->rz_next = trz;
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

// The Jacobi-PCG update; bj: then the element-interior blocks of the
// block-Jacobi preconditioner, which complete z and r.z and advance.
static int pcg_update_launch(const bs_problem *P, double *x, int init, cudaStream_t s,
                             bool bj = false) {
  CgVecs v = vecs(P);
  auto kern = k_pcg_update<1>;
  int grid = stream_grid(P->map->NG, 2, kReduceBlock, blocks_per_sm(kern, kReduceBlock));
  if (grid > kMaxPartials / 2) grid = kMaxPartials / 2;
  kern<<<grid, kReduceBlock, 0, s>>>(P->map->NG, v.p, v.Ap, v.dinv, x, v.r, v.z, P->d_partials,
                                     P->d_counter, P->d_state, init, bj ? 1 : 0);
  BS_LAUNCH_CHECK();
  if (bj) return bj_apply(P, v.r, v.dinv, v.z, init, s);
  return BS_OK;
}

// ------------------------------------------------------------ scattered storage

// owner[l] = 1 when l is the lowest local copy of its global node.
// NG, nnz: bounds of the checked build's index tests.
__global__ void k_owner(int64_t NL, int64_t NG, int64_t nnz, const int32_t *__restrict__ ids,
                        const int32_t *__restrict__ rs, const int32_t *__restrict__ cols,
                        uint8_t *__restrict__ owner) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t l = tid; l < NL; l += nth) {
    int32_t id = ids[l];
    if (!chk(bs_pred_map_entry(id, NG), BS_CHK_SCATTER_ENTRY) ||
        (id >= 0 && !chk(bs_pred_index(rs[id], nnz), BS_CHK_GATHER_ROW)))
      id = -1;
    owner[l] = id >= 0 && cols[rs[id]] == (int32_t)l ? 1 : 0;
  }
}

// xG[g] = xL at the lowest copy of g (0 for a node without copies).
__global__ void k_extract(int64_t NG, int64_t NL, int64_t nnz, const int32_t *__restrict__ rs,
                          const int32_t *__restrict__ cols, const double *__restrict__ xL,
                          double *__restrict__ xG) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = tid; g < NG; g += nth) {
    const int32_t a = rs[g];
    bool ok = a < rs[g + 1];
    if (ok && !chk(bs_pred_index(a, nnz) && bs_pred_index(cols[a], NL), BS_CHK_GATHER_COL))
      ok = false;
    xG[g] = ok ? xL[cols[a]] : 0.0;
  }
}

// qL[l] = qG[ids[l]] for unmasked l (BS7), and ep(sum over owned l of
// w[l] qL[l]).  Two consecutive local nodes per thread (8-byte map loads,
// 16-byte vector accesses; the vectors are 16-byte aligned), the odd last
// one by the first thread.
template <class Ep>
__global__ void __launch_bounds__(kReduceBlock)
    k_scatter_dot(int64_t NL, int64_t NG, const int32_t *__restrict__ ids,
                  const uint8_t *__restrict__ owner,
                  const double *__restrict__ qG, double *__restrict__ qL,
                  const double *__restrict__ w, double *partials, unsigned int *counter, Ep ep,
                  const CgState *st) {
  if (cg_halted(st)) return;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  const int64_t npair = NL / 2;
  for (int64_t q = tid; q < npair; q += nth) {
    int2 id = __ldcs(reinterpret_cast<const int2 *>(ids) + q);
    if (!chk(bs_pred_map_entry(id.x, NG), BS_CHK_SCATTER_ENTRY)) id.x = -1;
    if (!chk(bs_pred_map_entry(id.y, NG), BS_CHK_SCATTER_ENTRY)) id.y = -1;
    const uchar2 o = __ldcs(reinterpret_cast<const uchar2 *>(owner) + q);
    // a masked entry keeps its value: read the pair only when there is one
    double2 v = (id.x < 0 || id.y < 0) ? __ldcs(reinterpret_cast<const double2 *>(qL) + q)
                                       : make_double2(0.0, 0.0);
    if (id.x >= 0) v.x = __ldg(qG + id.x);
    if (id.y >= 0) v.y = __ldg(qG + id.y);
    __stcs(reinterpret_cast<double2 *>(qL) + q, v);
    if (o.x | o.y) {
      const double2 wv = __ldcs(reinterpret_cast<const double2 *>(w) + q);
      if (o.x) acc = fma(wv.x, v.x, acc);
      if (o.y) acc = fma(wv.y, v.y, acc);
    }
  }
  if ((NL & 1) && tid == 0) {
    const int64_t l = NL - 1;
    int32_t id = ids[l];
    if (!chk(bs_pred_map_entry(id, NG), BS_CHK_SCATTER_ENTRY)) id = -1;
    if (id >= 0) {
      const double v = qG[id];
      qL[l] = v;
      if (owner[l]) acc = fma(w[l], v, acc);
    }
  }
  const double part = block_sum<kReduceBlock>(acc);
  double total;
  if (grid_combine<kReduceBlock>(part, partials, counter, &total) && threadIdx.x == 0) ep(total);
}

// x += alpha p; r -= alpha Ap (skipped when init); JAC: z = dinv r; r.r and
// r.z over owned l; then the step of Algorithm 1 (or, init, r_0.r_0 and the
// stop flag after k_set_state).
template <bool JAC>
__global__ void __launch_bounds__(kReduceBlock)
    k_cg_update_L(int64_t NL, const double *__restrict__ p, const double *__restrict__ Ap,
                  const double *__restrict__ dinv, double *__restrict__ x,
                  double *__restrict__ r, double *__restrict__ z,
                  const uint8_t *__restrict__ owner, double *partials, unsigned int *counter,
                  CgState *st, int init) {
  if (!init && cg_halted(st)) return;
  const double alpha = init ? 0.0 : st->alpha;
  const double nalpha = -alpha;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  double rr = 0.0, rz = 0.0;
  auto one = [&](double &xi, double &ri, double pi, double Api, double di, double &zi, bool own) {
    if (!init) {
      xi = fma(alpha, pi, xi);
      ri = fma(nalpha, Api, ri);
    }
    if (JAC) zi = ri * di;
    if (own) {
      rr = fma(ri, ri, rr);
      if (JAC) rz = fma(ri, zi, rz);
    }
  };
  const int64_t npair = NL / 2;
  for (int64_t q = tid; q < npair; q += nth) {
    const uchar2 o = __ldcs(reinterpret_cast<const uchar2 *>(owner) + q);
    double2 xv = init ? make_double2(0.0, 0.0) : __ldcs(reinterpret_cast<const double2 *>(x) + q);
    double2 rv = __ldcs(reinterpret_cast<const double2 *>(r) + q);
    const double2 pv =
        init ? make_double2(0.0, 0.0) : __ldcs(reinterpret_cast<const double2 *>(p) + q);
    const double2 av =
        init ? make_double2(0.0, 0.0) : __ldcs(reinterpret_cast<const double2 *>(Ap) + q);
    const double2 dv =
        JAC ? __ldcs(reinterpret_cast<const double2 *>(dinv) + q) : make_double2(0.0, 0.0);
    double2 zv = make_double2(0.0, 0.0);
    one(xv.x, rv.x, pv.x, av.x, dv.x, zv.x, o.x != 0);
    one(xv.y, rv.y, pv.y, av.y, dv.y, zv.y, o.y != 0);
    if (!init) {
      __stcs(reinterpret_cast<double2 *>(x) + q, xv);
      __stcs(reinterpret_cast<double2 *>(r) + q, rv);
    }
    if (JAC) __stcs(reinterpret_cast<double2 *>(z) + q, zv);
  }
  if ((NL & 1) && tid == 0) {
    const int64_t l = NL - 1;
    double xi = x[l], ri = r[l], zi = 0.0;
    one(xi, ri, init ? 0.0 : p[l], init ? 0.0 : Ap[l], JAC ? dinv[l] : 0.0, zi, owner[l] != 0);
    if (!init) {
      x[l] = xi;
      r[l] = ri;
    }
    if (JAC) z[l] = zi;
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
    } else if (JAC) {
      const double beta = trz / st->rz;
      st->rz = trz;
      cg_advance(st, trr, beta);
    } else {
      cg_advance(st, trr, trr / st->rr);
    }
  }
}

struct LVecs {
  double *r, *p, *Ap, *x, *z, *dinv;
};
// Vector stride: N_L + 2 rounded up to even, so that every vector starts on
// a 16-byte boundary for the kernels' double2 accesses (N_L is odd for even N
// and an odd element count).
static int64_t lstride(const bs_map *m) { return (m->NL + 3) & ~(int64_t)1; }
static LVecs lvecs(const bs_problem *P) {
  const int64_t s = lstride(P->map);
  double *b = P->d_Lvec;
  return LVecs{b, b + s, b + 2 * s, b + 3 * s, b + 4 * s, b + 5 * s};
}

// The scattered vectors and the owner mask, on first use.
static int ensure_scattered(bs_problem *P, cudaStream_t s) {
  if (P->d_Lvec) return BS_OK;
  const bs_map *m = P->map;
  const int64_t n = 6 * lstride(m);
  cudaError_t e = cudaMalloc(&P->d_Lvec, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&P->d_owner, (size_t)m->NL + 16);
  if (e != cudaSuccess) {
    cudaFree(P->d_Lvec);
    cudaFree(P->d_owner);
    P->d_Lvec = nullptr;
    P->d_owner = nullptr;
    return fail(BS_ERR_ALLOC, "scattered CG: %s", cudaGetErrorString(e));
  }
  if (m->NL > 0) {
    k_owner<<<stream_grid(m->NL, 1, kStreamBlock, 8), kStreamBlock, 0, s>>>(
        m->NL, m->NG, m->nnz, m->d_ids, m->d_row_starts, m->d_col_ids, P->d_owner);
    BS_LAUNCH_CHECK();
  }
  return BS_OK;
}

static int update_L_launch(const bs_problem *P, bool precond, int init, cudaStream_t s) {
  LVecs L = lvecs(P);
  const int64_t NL = P->map->NL;
  auto launch = [&](auto kern) -> int {
    int grid = stream_grid(NL / 2 + 1, 1, kReduceBlock, blocks_per_sm(kern, kReduceBlock));
    if (grid > kMaxPartials / 2) grid = kMaxPartials / 2;
    kern<<<grid, kReduceBlock, 0, s>>>(NL, L.p, L.Ap, L.dinv, L.x, L.r, L.z, P->d_owner,
                                       P->d_partials, P->d_counter, P->d_state, init);
    BS_LAUNCH_CHECK();
    return BS_OK;
  };
  return precond ? launch(k_cg_update_L<true>) : launch(k_cg_update_L<false>);
}

// One scattered-storage iteration (five launches, see the top of the file).
static int scat_iteration(const bs_problem *P, bool precond, bool ff, cudaStream_t s) {
  const bs_map *m = P->map;
  CgVecs v = vecs(P);
  LVecs L = lvecs(P);
  CgState *st = P->d_state;
  const double g = 0.5 * P->h, mlam = P->lambda * g * g * g;
  int rc = P->d_geo
               ? (ff ? launch_ax_geo_ff<false>(P->N, m->E, m->NL, nullptr, nullptr, L.p,
                                               P->d_ApL, P->d_tabff, P->d_coef, P->d_geo,
                                               P->lambda, st, s)
                     : launch_ax_geo<false>(P->N, m->E, m->NL, nullptr, nullptr, L.p, P->d_ApL,
                                            P->d_tab, P->d_coef, P->d_geo, P->lambda, st, s))
           : ff ? launch_ax_local_ff<false>(P->N, m->E, nullptr, nullptr, L.p, P->d_ApL,
                                            P->d_tabff, P->d_coef, g, mlam, st, s)
                : launch_ax_local<double, false>(P->N, m->E, nullptr, nullptr, L.p, P->d_ApL,
                                                 P->d_tab, P->d_coef, g, mlam, st, s);
  if (!rc)
    rc = launch_gather<double, false, EpNone>(m, P->d_ApL, v.Ap, nullptr, nullptr, nullptr,
                                              EpNone{}, st, s);
  if (rc) return rc;
  {
    auto kern = k_scatter_dot<EpAlpha>;
    int grid = stream_grid(m->NL / 2 + 1, 1, kReduceBlock, blocks_per_sm(kern, kReduceBlock));
    if (grid > kMaxPartials) grid = kMaxPartials;
    kern<<<grid, kReduceBlock, 0, s>>>(m->NL, m->NG, m->d_ids, P->d_owner, v.Ap, L.Ap, L.p,
                                       P->d_partials, P->d_counter,
                                       EpAlpha{st, precond ? 1 : 0}, st);
    BS_LAUNCH_CHECK();
  }
  if ((rc = update_L_launch(P, precond, 0, s))) return rc;
  return launch_axpy<double>(m->NL, Scalar<double>{1.0, nullptr}, precond ? L.z : L.r,
                             Scalar<double>{0.0, &st->beta}, L.p, st, s);
}

// r_L = Z r_G (r_G = b - A x0 already in the global r), x_L = Z x0 or 0,
// Jacobi's dinv_L = Z dinv_G, then r_0.r_0 (and z_0, r_0.z_0) and p_0.
static int scat_setup(bs_problem *P, const double *x, bool x0, bool precond, double tol,
                      int maxit, bool fixed, double *d_hist, cudaStream_t s) {
  const bs_map *m = P->map;
  CgVecs v = vecs(P);
  if (int rc = ensure_scattered(P, s)) return rc;
  LVecs L = lvecs(P);
  BS_CUDA_TRY(cudaMemsetAsync(P->d_Lvec, 0, sizeof(double) * 6 * lstride(m), s));
  if (m->NL > 0) {
    if (int rc = launch_scatter<double>(m, v.r, L.r, s)) return rc;
    if (x0)
      if (int rc = launch_scatter<double>(m, x, L.x, s)) return rc;
    if (precond)
      if (int rc = launch_scatter<double>(m, v.dinv, L.dinv, s)) return rc;
  }
  k_set_state<<<1, 1, 0, s>>>(P->d_state, tol * tol, maxit, fixed ? 1 : 0, d_hist);
  BS_CUDA_TRY(cudaGetLastError());
  if (int rc = update_L_launch(P, precond, 1, s)) return rc;
  return launch_copy<double>(m->NL, precond ? L.z : L.r, L.p, s);
}

// One CG iteration (four launches: the operator with p.Ap, the fused update
// with r.r, the direction).  ff: the float-float element operator.
static int cg_iteration(const bs_problem *P, double *x, bool precond, bool ff, cudaStream_t s,
                        bool bj = false) {
  const bs_map *m = P->map;
  CgVecs v = vecs(P);
  CgState *st = P->d_state;
  const double g = 0.5 * P->h, mlam = P->lambda * g * g * g;
  int rc = apply_A_global<double, true, EpAlpha>(P, ff, P->d_tab, v.p, v.Ap, P->d_ApL, g, mlam,
                                                 EpAlpha{st, precond ? 1 : 0}, st, s);
  if (rc) return rc;
  if (precond) {
    rc = pcg_update_launch(P, x, 0, s, bj);
  } else {
    rc = launch_cg_update<double, EpBeta>(m->NG, Scalar<double>{0.0, &st->alpha}, v.p, v.Ap, x,
                                          v.r, P->d_partials, P->d_counter, EpBeta{st}, st, s);
  }
  if (rc) return rc;
  return launch_axpy<double>(m->NG, Scalar<double>{1.0, nullptr}, precond ? v.z : v.r,
                             Scalar<double>{0.0, &st->beta}, v.p, st, s);
}

static int capture_chunk(bs_problem *P, double *x, bool precond, bool ff, bool scat,
                         int chunk, bool bj = false) {
  const void *key[4] = {x, (const void *)(intptr_t)((precond ? 1 : 0) | (ff ? 2 : 0) |
                                                     (g_op_fusion ? 4 : 0) | (scat ? 8 : 0) |
                                                     (g_op_evenodd ? 16 : 0) | (bj ? 32 : 0)),
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
  for (int c = 0; c < chunk && rc == BS_OK; ++c)
    rc = scat ? scat_iteration(P, precond, ff, cs) : cg_iteration(P, x, precond, ff, cs, bj);
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
  const bool bj = flags & BS_CG_BLOCK_JACOBI;
  const bool precond = (flags & BS_CG_JACOBI) || bj;
  const bool ff = flags & BS_CG_FF_OPERATOR;
  const bool scat = flags & BS_CG_SCATTERED;
  BS_ARG(!bj || (!scat && !P->d_geo && P->N >= 2 && P->N <= kBjMaxNi + 1),
         "bs_cg_solve: BS_CG_BLOCK_JACOBI needs affine elements of degree 2..9 in global "
         "storage");
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
    }
    if (scat) {
      BS_TRY(scat_setup(P, x, flags & BS_CG_X0, precond, tol, maxit, fixed, d_hist, s));
    } else if (precond) {
      if (bj) BS_TRY(bj_ensure(P, s));
      k_set_state<<<1, 1, 0, s>>>(st, tol * tol, maxit, fixed ? 1 : 0, d_hist);
      BS_TRY(pcg_update_launch(P, x, 1, s, bj));  // z = M^-1 r, rr, rz, stop flag
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
    if (graph && maxit > 0) BS_TRY(capture_chunk(P, x, precond, ff, scat, chunk, bj));
    while (launched < maxit) {
      if (graph) {
        BS_CUDA_TRY(cudaGraphLaunch(P->graph, s));
      } else {
        for (int c = 0; c < chunk; ++c)
          BS_TRY(scat ? scat_iteration(P, precond, ff, s)
                      : cg_iteration(P, x, precond, ff, s, bj));
      }
      launched += chunk;
      BS_CUDA_TRY(cudaMemcpyAsync(P->h_state, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
      BS_CUDA_TRY(cudaStreamSynchronize(s));
      if (P->h_state->done) break;
    }
    if (scat && NG > 0) {  // x_G from the lowest copy of each node
      k_extract<<<stream_grid(NG, 1, kStreamBlock, 8), kStreamBlock, 0, s>>>(
          NG, m->NL, m->nnz, m->d_row_starts, m->d_col_ids, lvecs(P).x, x);
      BS_CUDA_TRY(cudaGetLastError());
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
