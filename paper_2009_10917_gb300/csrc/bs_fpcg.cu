// bs_fpcg.cu -- flexible PCG with the learned element preconditioner, and
// the extraction of its training pairs.
//
// Preconditioner (no counterpart in the paper):
//   u = Z (D^-1 r);  rms_e = sqrt(mean of u_e^2);  X_e = u_e / rms_e
//   Y = W2 relu(W1 X), or the odd part W2 W1 X / 2, at the element-interior
//       outputs only (tensor-core GEMMs over all elements at once, in the
//       network's BF16 or BF16x3 mode; the odd part is one GEMM with
//       L = W2 W1 / 2)
//   z = D^-1 r + corr, corr_g = rms_e Y_e,l at the interior node g of element
//       e (local index l), 0 elsewhere
// The training targets are the element-interior error, zero at every other
// node, so only interior outputs are used; interior nodes belong to one
// element each, so the GEMM epilogue writes them straight into corr (no
// gather).  Flexible CG (Polak-Ribiere): alpha = r.z / p.Ap; x += alpha p;
// r -= alpha Ap; z' = M(r), replaced by D^-1 r when r.z' <= 0 or not finite
// (the Jacobi fallback); beta = r.(z' - z) / (r.z)_old; p = z' + beta p.
// Every scalar and the fallback decision are formed on the device; an
// iteration is seven launches (six for Jacobi-only) and never waits for the
// host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "bs_mlp.cuh"
#include "bs_op_ff.cuh"

namespace bs {

constexpr int kPrepBlock = 256;  // 8 warps, one element per warp

// One warp per element: u = D^-1 r through the map, rms, the X row as the
// GEMM operand ([hi] or [hi | hi | lo], padding zero), and rms * oscale to
// rmsv[e] in double (0 for an all-zero element).  GB300's FP64 pipe (and the
// conversions, which share it) runs at 1/64 of the FP32 rate, so no node
// touches it: r and D^-1 are brought to [1, 2) relative to their largest
// value in the element by an exponent shift and truncated to their 24-bit
// high parts, all by integer operations (relative error below 2^-23 each);
// u, the sum of squares and the scaling are FP32, and the shift is added
// back to rms, in double, once per element.  Values more than 2^-126 below
// the element's largest count as zero.  rms is only a normalisation: the
// network's output is multiplied back by the same value.
constexpr int kPrepMaxNq = 10;  // degrees up to 9

// Biased exponent of a double (0 for zero and subnormals).
__device__ __forceinline__ int dexp(double x) {
  return ((unsigned)__double2hiint(x) >> 20) & 0x7ff;
}
// x 2^(1023 - emax), truncated to 24 significant bits, as a float; 0 when
// that is below 2^-126 (or x is zero or subnormal).
__device__ __forceinline__ float shifted_hi(double x, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const int E = (int)((hw >> 20) & 0x7ffu);
  const int fe = E - emax + 127;  // float exponent field of the shifted value
  if (E == 0 || fe < 1) return 0.f;
  return __uint_as_float((hw & 0x80000000u) | ((unsigned)fe << 23) | ((hw & 0xfffffu) << 3) |
                         (lw >> 29));
}

template <int NP>
__global__ void __launch_bounds__(kPrepBlock)
    k_fp_prep(int64_t E, int64_t NG, int Dp, int split, float oscale,
              const int32_t *__restrict__ order,
              const int32_t *__restrict__ ids, const double *__restrict__ r,
              const double *__restrict__ dinv, __nv_bfloat16 *__restrict__ X,
              double *__restrict__ rmsv, const CgState *st) {
  constexpr int T = (NP + 31) / 32;  // nodes per lane
  if (cg_halted(st)) return;
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * (kPrepBlock / 32) + (threadIdx.x >> 5);
  if (q >= E) return;
  const int64_t e = order[q];
  if (!chk(bs_pred_index(e, E), BS_CHK_PREC_ENTRY)) return;  // warp-uniform
  const int32_t *id = ids + e * NP;
  // all of a lane's map entries, then all of its gathers, so that the loads
  // of an element are in flight together
  int32_t g[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int l = lane + 32 * t;
    g[t] = l < NP ? __ldcs(id + l) : -1;
    if (!chk(bs_pred_map_entry(g[t], NG), BS_CHK_PREC_ENTRY)) g[t] = -1;
  }
  double rv[T], dv[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    rv[t] = g[t] >= 0 ? __ldg(r + g[t]) : 0.0;
    dv[t] = g[t] >= 0 ? __ldg(dinv + g[t]) : 0.0;
  }
  int er = 0, ed = 0;  // largest exponents in the element
#pragma unroll
  for (int t = 0; t < T; ++t) {
    er = max(er, dexp(rv[t]));
    ed = max(ed, dexp(dv[t]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    er = max(er, __shfl_xor_sync(0xffffffffu, er, o));
    ed = max(ed, __shfl_xor_sync(0xffffffffu, ed, o));
  }
  float uf[T];
  float ss = 0.f;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    uf[t] = shifted_hi(dv[t], ed) * shifted_hi(rv[t], er);
    ss = fmaf(uf[t], uf[t], ss);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const float rms = sqrtf(ss / (float)NP);
  const float inv = rms > 0.f ? 1.0f / rms : 0.f;
  __nv_bfloat16 *row = X + q * (split ? 3 * Dp : Dp);
#pragma unroll
  for (int t = 0; t < (T > 0 ? T : 1) + 1; ++t) {  // Dp may exceed 32 T by up to 31
    const int l = lane + 32 * t;
    if (l >= Dp) break;
    __nv_bfloat16 hi, lo;
    bf16_split(t < T && l < NP ? uf[t < T ? t : 0] * inv : 0.f, hi, lo);
    row[l] = hi;
    if (split) {
      row[Dp + l] = hi;
      row[2 * Dp + l] = lo;
    }
  }
  // the true rms: undo the two shifts (2^(er - 1023) and 2^(ed - 1023))
  if (lane == 0) rmsv[q] = rms > 0.f ? ldexp((double)(rms * oscale), er + ed - 2046) : 0.0;
}

static int launch_fp_prep(int N, int64_t E, int64_t NG, int Dp, int split, float oscale,
                          const int32_t *order,
                          const int32_t *ids, const double *r, const double *dinv,
                          __nv_bfloat16 *X, double *rmsv, const CgState *st, cudaStream_t s) {
  const unsigned grid = (unsigned)((E + kPrepBlock / 32 - 1) / (kPrepBlock / 32));
#define BS_PREP_CASE(NQ)                                                                     \
  case NQ:                                                                                   \
    k_fp_prep<NQ * NQ * NQ><<<grid, kPrepBlock, 0, s>>>(E, NG, Dp, split, oscale, order, ids, \
                                                        r, dinv, X, rmsv, st);               \
    break;
  switch (N + 1) {
    BS_PREP_CASE(3)
    BS_PREP_CASE(4)
    BS_PREP_CASE(5)
    BS_PREP_CASE(6)
    BS_PREP_CASE(7)
    BS_PREP_CASE(8)
    BS_PREP_CASE(9)
    BS_PREP_CASE(10)
    default:
      return fail(BS_ERR_ARG, "learned FPCG: degree %d outside 2..9", N);
  }
#undef BS_PREP_CASE
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// Three-value last-block-done combine (partials holds 3 * gridDim.x).
template <int BLOCK>
__device__ __forceinline__ bool grid_combine3(double a, double b, double c, double *partials,
                                              unsigned int *counter, double *ta, double *tb,
                                              double *tc) {
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x] = a;
    partials[3 * blockIdx.x + 1] = b;
    partials[3 * blockIdx.x + 2] = c;
    __threadfence();
    s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double va = 0.0, vb = 0.0, vc = 0.0;
  for (unsigned int k = threadIdx.x; k < gridDim.x; k += BLOCK) {
    va = va + __ldcg(partials + 3 * k);
    vb = vb + __ldcg(partials + 3 * k + 1);
    vc = vc + __ldcg(partials + 3 * k + 2);
  }
  va = block_sum<BLOCK>(va);
  vb = block_sum<BLOCK>(vb);
  vc = block_sum<BLOCK>(vc);
  if (threadIdx.x == 0) {
    *ta = va;
    *tb = vb;
    *tc = vc;
    *counter = 0u;
  }
  return true;
}

// After z' is formed: rzn = r.z', rzo = r.z_old, rzj = r.(D^-1 r).  Decides
// the fallback, beta (Polak-Ribiere) and the new r.z.  init: first z, no beta.
__device__ void fpcg_scalars(CgState *st, double rzn, double rzo, double rzj, int init) {
  int fb = 0;
  if (!(rzn > 0.0) || !isfinite(rzn)) {
    fb = 1;
    rzn = rzj;
  }
  st->fallback = fb;
  st->nfallback += fb;
  if (!init) {
    const double beta = (rzn - rzo) / st->rz;
    st->beta = beta;
    if (!isfinite(beta)) st->done = 2;
  } else {
    st->beta = 0.0;
  }
  st->rz = rzn;
}

// z' = D^-1 r + corr (have_mlp) or D^-1 r, with the three dot products
// r.z', r.z_old, r.(D^-1 r); z holds the old z on entry and z' on exit.  z'
// is one FP64 fused multiply-add per node; the dot products run on the FP32
// pipes as float-pair sums of exact float-pair splits (error a few units of
// 2^-46 of the sum of |terms|), falling back to FP64 for values outside
// [2^-60, 2^60), so the kernel is bound by HBM, not by GB300's narrow FP64
// pipe, at any scale of the data.
__global__ void __launch_bounds__(kReduceBlock)
    k_fpcg_z(int64_t NG, const double *__restrict__ r, const double *__restrict__ dinv,
             const double *__restrict__ corr, double *__restrict__ z, double *partials,
             unsigned int *counter, CgState *st, int init, int have_mlp) {
  if (cg_halted(st)) return;
  FF an{0.f, 0.f}, ao{0.f, 0.f}, aj{0.f, 0.f};
  double dn = 0.0, dlo = 0.0, dj = 0.0;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = tid; g < NG; g += nth) {
    const double rg = r[g], dg = dinv[g];
    const double zj = dg * rg;
    const double zn = have_mlp ? fma(dg, rg, corr[g]) : zj;
    if (!init) ff_dot_acc(ao, dlo, rg, z[g]);
    ff_dot_acc(an, dn, rg, zn);
    ff_dot_acc(aj, dj, rg, zj);
    z[g] = zn;
  }
  const double pn = block_sum<kReduceBlock>(ff_widen(an.hi) + ff_widen(an.lo) + dn);
  const double po = block_sum<kReduceBlock>(ff_widen(ao.hi) + ff_widen(ao.lo) + dlo);
  const double pj = block_sum<kReduceBlock>(ff_widen(aj.hi) + ff_widen(aj.lo) + dj);
  double tn, to, tj;
  if (grid_combine3<kReduceBlock>(pn, po, pj, partials, counter, &tn, &to, &tj) &&
      threadIdx.x == 0)
    fpcg_scalars(st, tn, to, tj, init);
}

// p = z' + beta p, with z' = D^-1 r (stored back) when the correction fell back.
__global__ void k_fpcg_dir(int64_t n, const double *__restrict__ r, const double *__restrict__ dinv,
                           double *__restrict__ z, double *__restrict__ p, const CgState *st) {
  if (cg_halted(st)) return;
  const int fb = st->fallback;
  const double beta = st->beta;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += nth) {
    double zi = z[i];
    if (fb) {
      zi = dinv[i] * r[i];
      z[i] = zi;
    }
    p[i] = fma(beta, p[i], zi);
  }
}

struct EpAlphaRz {  // p.Ap -> alpha = r.z / p.Ap
  CgState *st;
  __device__ __forceinline__ void operator()(double s) const {
    st->pAp = s;
    if (!(s > 0.0) || !isfinite(s)) {
      st->done = 2;
      return;
    }
    st->alpha = st->rz / s;
  }
};

struct EpResidual {  // r.r after the update: stop rule
  CgState *st;
  __device__ __forceinline__ void operator()(double s) const {
    const int j = st->iter;
    if (st->hist) {
      st->hist[3 * j] = st->alpha;
      st->hist[3 * j + 1] = st->beta;
      st->hist[3 * j + 2] = s;
    }
    st->rr = s;
    st->iter = j + 1;
    if (!isfinite(s))
      st->done = 2;
    else if (s <= st->eps)
      st->done = 1;
    else if (j + 1 >= st->maxit)
      st->done = 3;
  }
};

struct EpBbF {  // b.b
  CgState *st;
  __device__ __forceinline__ void operator()(double s) const { st->bb = s; }
};

__global__ void k_fpcg_init(CgState *st, double tol2, int maxit) {
  st->nfallback = 0;
  st->fallback = 0;
  st->eps = tol2 * st->bb;
  st->rr = st->bb;  // r_0 = b
  st->iter = 0;
  st->maxit = maxit;
  st->fixed = 0;
  st->hist = nullptr;
  st->alpha = st->beta = 0.0;
  st->done = !isfinite(st->bb) ? 2 : (st->bb <= st->eps ? 1 : (maxit <= 0 ? 3 : 0));
}

__global__ void k_recip(int64_t n, const double *__restrict__ d, double *__restrict__ inv) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += nth) inv[i] = 1.0 / d[i];
}

struct FpVecs {
  double *r, *p, *Ap, *z, *dinv, *corr;
};
static FpVecs fpvecs(const bs_problem *P) {
  const int64_t s = P->map->NG + 2;
  double *v = P->d_vec;
  return FpVecs{v, v + s, v + 2 * s, v + 3 * s, v + 4 * s, v + 5 * s};
}

// z' = M(r) into v.z (with the dots and beta); init: the first z.
static int precondition(const bs_problem *P, bs_mlp *mlp, int odd, int init, cudaStream_t s) {
  const bs_map *m = P->map;
  FpVecs v = fpvecs(P);
  CgState *st = P->d_state;
  const int Np = (P->N + 1) * (P->N + 1) * (P->N + 1);
  if (mlp) {
    const int64_t E = m->E;
    double *rmsv = reinterpret_cast<double *>(mlp->Y);  // E doubles of inference scratch
    if (int rc = launch_fp_prep(P->N, E, m->NG, mlp->Dp, mlp->split, 1.0f, m->d_elem_order,
                                m->d_ids, v.r, v.dinv, mlp->Xb, rmsv, st, s))
      return rc;
    GemmArgs b{};
    b.nvalid = mlp->nI;
    b.out_f64 = v.corr;
    b.scale = rmsv;
    b.ids = m->d_ids;
    b.order = m->d_elem_order;
    b.lidx = mlp->lidx;
    b.np = Np;
    b.ng = m->NG;
    b.st = st;
    if (odd) {
      // the odd part W2 W1 x / 2 is linear: one GEMM with the interior rows of
      // L = W2 W1 / 2
      const int K1 = mlp->split ? 3 * mlp->Dp : mlp->Dp;
      b.A = mlp->Xb;
      b.B = mlp->Wint;
      b.M = E;
      b.N = mlp->nI;
      b.K = K1;
      b.lda = K1;
      b.ldb = K1;
      if (int rc = launch_gemm(EPI_SCATTER_F64, b, s)) return rc;
    } else {
      // hidden layer over all H units, then the interior rows of W2
      const int K1 = mlp->split ? 3 * mlp->Dp : mlp->Dp, K2 = mlp->split ? 3 * mlp->H : mlp->H;
      GemmArgs a{};
      a.A = mlp->Xb;
      a.B = mlp->W1b;
      a.M = E;
      a.N = mlp->H;
      a.K = K1;
      a.lda = K1;
      a.ldb = K1;
      a.ldc = K2;
      a.out_b16 = mlp->Hb;
      a.relu = 1;
      a.split = mlp->split ? mlp->H : 0;
      a.st = st;
      if (int rc = launch_gemm(EPI_HIDDEN, a, s)) return rc;
      b.A = mlp->Hb;
      b.B = mlp->Wint;
      b.M = E;
      b.N = mlp->nI;
      b.K = K2;
      b.lda = K2;
      b.ldb = K2;
      if (int rc = launch_gemm(EPI_SCATTER_F64, b, s)) return rc;
    }
  }
  int grid = stream_grid(m->NG, 1, kReduceBlock, blocks_per_sm(k_fpcg_z, kReduceBlock));
  if (grid > kMaxPartials / 3) grid = kMaxPartials / 3;
  k_fpcg_z<<<grid, kReduceBlock, 0, s>>>(m->NG, v.r, v.dinv, v.corr, v.z, P->d_partials,
                                         P->d_counter, st, init, mlp ? 1 : 0);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

static int fpcg_iteration(const bs_problem *P, bs_mlp *mlp, int odd, bool ff, double *x,
                          cudaStream_t s) {
  const bs_map *m = P->map;
  FpVecs v = fpvecs(P);
  CgState *st = P->d_state;
  const double g = 0.5 * P->h, mlam = P->lambda * g * g * g;
  int rc = apply_A_global<double, true, EpAlphaRz>(P, ff, P->d_tab, v.p, v.Ap, P->d_ApL, g,
                                                   mlam, EpAlphaRz{st}, st, s);
  if (!rc)
    rc = launch_cg_update<double, EpResidual>(m->NG, Scalar<double>{0.0, &st->alpha}, v.p, v.Ap,
                                              x, v.r, P->d_partials, P->d_counter,
                                              EpResidual{st}, st, s);
  if (!rc) rc = precondition(P, mlp, odd, 0, s);
  if (rc) return rc;
  k_fpcg_dir<<<stream_grid(m->NG, 1, 256, 8), 256, 0, s>>>(m->NG, v.r, v.dinv, v.z, v.p, st);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// Sum over a block of up to 4 warps (every thread calls; result to all).
__device__ __forceinline__ double small_block_sum(double v, double *s_red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = v + __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();  // s_red may still be read by a previous call
  if ((threadIdx.x & 31) == 0) s_red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < nw; ++k) t = t + s_red[k];
  return t;
}

// Training pairs: one block per pair q, one thread per column (i, j) of
// element e = elems[q].  u = D^-1 r on the element; the interior error e_I
// solves A_II e_I = r_I by Jacobi-preconditioned CG in shared memory (the
// element operator applied with the other nodes held at zero), to
// r.r <= 1e-26 r_0.r_0 or 4 n_I iterations.  Rows X[q] = s u / rms,
// T[q] = s (e_I - u_I) / rms on interior nodes, 0 elsewhere.
template <int NQ>
__global__ void __launch_bounds__(128)
    k_interior_pairs(int64_t count, const int32_t *__restrict__ elems,
                     const int32_t *__restrict__ ids, const double *__restrict__ r,
                     const double *__restrict__ dinv, const OpTab<double> *__restrict__ tab,
                     const double *__restrict__ coef, double g, double mlam, int negate_odd,
                     float *__restrict__ X, float *__restrict__ T) {
  constexpr int NP = NQ * NQ * NQ, NQ2 = NQ * NQ, N = NQ - 1;
  __shared__ double s_u[NP], s_p[NP], s_res[NP], s_x[NP], s_d[NP];
  __shared__ double s_K[NQ2], s_w[NQ], s_red[4];
  const int64_t q = blockIdx.x;
  if (q >= count) return;
  const int t = threadIdx.x;
  for (int k = t; k < NQ2; k += blockDim.x) s_K[k] = tab->K[k];
  for (int k = t; k < NQ; k += blockDim.x) s_w[k] = tab->w[k];
  const int32_t e = elems[q];
  if (!chk(bs_pred_index(e, tab->ne), BS_CHK_PREC_ENTRY)) return;  // block-uniform
  const int32_t *id = ids + (int64_t)e * NP;
  const double c = coef ? coef[e] : 1.0;
  const double sgn = (negate_odd && (q & 1)) ? -1.0 : 1.0;
  const bool col = t < NQ2;
  const int i = t % NQ, j = t / NQ;
  double ss = 0.0;
  unsigned imask = 0u;  // bit k: node (i, j, k) is an unmasked interior node
  __syncthreads();
  if (col) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const int l = i + NQ * j + NQ2 * k;
      int32_t gI = id[l];
      if (!chk(bs_pred_map_entry(gI, tab->ng), BS_CHK_PREC_ENTRY)) gI = -1;
      const double u = gI >= 0 ? dinv[gI] * r[gI] : 0.0;
      s_u[l] = u;
      ss = fma(u, u, ss);
      const bool in = gI >= 0 && i >= 1 && i < N && j >= 1 && j < N && k >= 1 && k < N;
      imask |= (in ? 1u : 0u) << k;
      const double rv = in ? r[gI] : 0.0;
      s_res[l] = rv;
      s_x[l] = 0.0;
      // Jacobi diagonal of c S + lambda M at this node (1 off the interior)
      const double wi = s_w[i], wj = s_w[j], wk = s_w[k];
      const double dg = c * g * (s_K[i * NQ + i] * wj * wk + wi * s_K[j * NQ + j] * wk +
                                 wi * wj * s_K[k * NQ + k]) +
                        mlam * (wi * wj * wk);
      s_d[l] = in ? dg : 1.0;
      s_p[l] = in ? rv / dg : 0.0;  // p_0 = z_0 = D_I^-1 r_I
    }
  }
  const double rms = sqrt(small_block_sum(ss, s_red) / NP);
  float *xo = X + q * NP, *to = T + q * NP;
  if (!(rms > 0.0)) {
    for (int l = t; l < NP; l += blockDim.x) xo[l] = to[l] = 0.f;
    return;
  }
  double rz = 0.0, rr0 = 0.0;
  if (col)
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const int l = i + NQ * j + NQ2 * k;
      rz = fma(s_res[l], s_p[l], rz);
      rr0 = fma(s_res[l], s_res[l], rr0);
    }
  rz = small_block_sum(rz, s_red);
  rr0 = small_block_sum(rr0, s_red);
  const int maxit = 4 * (N - 1) * (N - 1) * (N - 1) + 4;
  double Ap[NQ];
  for (int it = 0; it < maxit && rr0 > 0.0; ++it) {
    // Ap = A_II p (p is zero off the interior)
    double pAp = 0.0;
    if (col) {
      const double wi = s_w[i], wj = s_w[j];
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        double ar = 0.0, as = 0.0, at = 0.0;
#pragma unroll
        for (int m = 0; m < NQ; ++m) {
          ar = fma(s_K[i * NQ + m], s_p[m + NQ * j + NQ2 * k], ar);
          as = fma(s_K[j * NQ + m], s_p[i + NQ * m + NQ2 * k], as);
          at = fma(s_K[k * NQ + m], s_p[i + NQ * j + NQ2 * m], at);
        }
        const double wk = s_w[k];
        const int l = i + NQ * j + NQ2 * k;
        const double stiff = (wj * wk) * ar + (wi * wk) * as + (wi * wj) * at;
        Ap[k] = ((imask >> k) & 1u) ? c * g * stiff + mlam * (wi * wj * wk) * s_p[l] : 0.0;
        pAp = fma(s_p[l], Ap[k], pAp);
      }
    }
    pAp = small_block_sum(pAp, s_red);
    if (!(pAp > 0.0)) break;
    const double alpha = rz / pAp;
    double rr = 0.0, rzn = 0.0;
    if (col)
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        const int l = i + NQ * j + NQ2 * k;
        s_x[l] = fma(alpha, s_p[l], s_x[l]);
        const double rv = fma(-alpha, Ap[k], s_res[l]);
        s_res[l] = rv;
        rr = fma(rv, rv, rr);
        rzn = fma(rv, rv / s_d[l], rzn);
      }
    rr = small_block_sum(rr, s_red);
    rzn = small_block_sum(rzn, s_red);
    if (rr <= 1e-26 * rr0) break;
    const double beta = rzn / rz;
    rz = rzn;
    if (col)
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        const int l = i + NQ * j + NQ2 * k;
        s_p[l] = fma(beta, s_p[l], s_res[l] / s_d[l]);
      }
    __syncthreads();
  }
  __syncthreads();
  const double inv = sgn / rms;
  for (int l = t; l < NP; l += blockDim.x) {
    const int a = l % NQ, b = (l / NQ) % NQ, k = l / NQ2;
    const bool in = a >= 1 && a < N && b >= 1 && b < N && k >= 1 && k < N && id[l] >= 0;
    xo[l] = (float)(s_u[l] * inv);
    to[l] = in ? (float)((s_x[l] - s_u[l]) * inv) : 0.f;
  }
}

static int fpcg_setup(const bs_problem *P, cudaStream_t s) {
  FpVecs v = fpvecs(P);
  const bs_map *m = P->map;
  if (int rc = bs_diag_A(P, v.Ap, s)) return rc;
  const int grid = stream_grid(m->NG, 1, 256, 8);
  k_recip<<<grid, 256, 0, s>>>(m->NG, v.Ap, v.dinv);
  BS_LAUNCH_CHECK();
  // corr is written only at element-interior nodes; the rest stays zero
  BS_CUDA_TRY(cudaMemsetAsync(v.corr, 0, sizeof(double) * m->NG, s));
  return BS_OK;
}

}  // namespace bs

using namespace bs;

extern "C" {

int bs_mlp_pairs(const bs_problem *P, const double *d_r, int64_t count, const int32_t *d_elems,
                 int32_t negate_odd, float *d_X, float *d_T, void *stream) {
  BS_ARG(P && P->map, "bs_mlp_pairs: problem is NULL");
  BS_ARG(count >= 0, "bs_mlp_pairs: count < 0");
  BS_ARG(!P->d_geo, "bs_mlp_pairs: not available with geometric factors");
  BS_ARG(P->N >= 2 && P->N <= 8, "bs_mlp_pairs: degree %d outside 2..8", P->N);
  if (count == 0) return BS_OK;
  BS_ARG(d_r && d_elems && d_X && d_T, "bs_mlp_pairs: NULL argument");
  BS_ARG(count <= 0x7fffffff, "bs_mlp_pairs: count too large");
  int dev = -1;
  BS_CUDA_TRY(cudaGetDevice(&dev));
  BS_ARG(dev == P->device, "bs_mlp_pairs: problem on another device");
  cudaStream_t s = as_stream(stream);
  if (int rc = fpcg_setup(P, s)) return rc;
  FpVecs v = fpvecs(P);
  const double g = 0.5 * P->h, mlam = P->lambda * g * g * g;
  const bs_map *m = P->map;
#define BS_PAIRS_CASE(NQ)                                                                   \
  case NQ:                                                                                  \
    k_interior_pairs<NQ><<<(unsigned)count, ((NQ * NQ + 31) / 32) * 32, 0, s>>>(            \
        count, d_elems, m->d_ids, d_r, v.dinv, P->d_tab, P->d_coef, g, mlam, negate_odd, d_X, \
        d_T);                                                                               \
    break;
  switch (P->N + 1) {
    BS_PAIRS_CASE(3)
    BS_PAIRS_CASE(4)
    BS_PAIRS_CASE(5)
    BS_PAIRS_CASE(6)
    BS_PAIRS_CASE(7)
    BS_PAIRS_CASE(8)
    BS_PAIRS_CASE(9)
    default: break;
  }
#undef BS_PAIRS_CASE
  BS_LAUNCH_CHECK();
  return BS_OK;
}

int bs_fpcg_learned(const bs_problem *Pc, bs_mlp *mlp, const double *b, double *x, double tol,
                    int32_t maxit, int32_t flags, bs_cg_info *info, void *stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (info) memset(info, 0, sizeof(*info));
  BS_ARG(Pc != nullptr, "bs_fpcg_learned: problem is NULL");
  bs_problem *P = const_cast<bs_problem *>(Pc);
  int dev = -1;
  BS_CUDA_TRY(cudaGetDevice(&dev));
  BS_ARG(dev == P->device, "bs_fpcg_learned: problem on another device");
  BS_ARG(!P->d_geo, "bs_fpcg_learned: not available with geometric factors");
  BS_ARG(maxit >= 0 && tol >= 0.0 && std::isfinite(tol), "bs_fpcg_learned: bad tol or maxit");
  BS_ARG((flags & ~(BS_CG_GRAPH | BS_FPCG_ODD | BS_FPCG_NO_JUDGE | BS_CG_FF_OPERATOR)) == 0,
         "bs_fpcg_learned: unknown flags 0x%x", (unsigned)flags);
  const bool ff = flags & BS_CG_FF_OPERATOR;
  const bool judge = !(flags & BS_FPCG_NO_JUDGE);
  const int odd = (flags & BS_FPCG_ODD) ? 1 : 0;
  const bs_map *m = P->map;
  const int Np = (P->N + 1) * (P->N + 1) * (P->N + 1);
  if (mlp) {
    BS_ARG(mlp->device == dev, "bs_fpcg_learned: mlp on another device");
    BS_ARG(mlp->D == Np, "bs_fpcg_learned: mlp input size %d != (N+1)^3 = %d", mlp->D, Np);
    BS_ARG(P->N + 1 <= kPrepMaxNq, "bs_fpcg_learned: degree %d above 9", P->N);
    if (int rc = mlp_ensure(mlp, m->E > 32 ? m->E : 32)) return rc;
    BS_ARG(mlp->nI > 0, "bs_fpcg_learned: the network needs N >= 2 (element-interior outputs)");
    if (int rc = mlp_interior_operand(mlp, odd, as_stream(stream))) return rc;
  }
  BS_ARG(m->NG == 0 || (b && x), "bs_fpcg_learned: NULL vector");
  cudaStream_t s = as_stream(stream);
  FpVecs v = fpvecs(P);
  CgState *st = P->d_state;
  int rc = fpcg_setup(P, s);
  if (rc) return rc;
  BS_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * m->NG, s));
  rc = launch_copy<double>(m->NG, b, v.r, s);
  if (!rc)
    rc = launch_dot<double, true, EpBbF>(m->NG, b, b, P->d_partials, P->d_counter, EpBbF{st},
                                        nullptr, s);
  if (rc) return rc;
  k_fpcg_init<<<1, 1, 0, s>>>(st, tol * tol, maxit);
  BS_LAUNCH_CHECK();
  BS_CUDA_TRY(cudaMemsetAsync(v.p, 0, sizeof(double) * m->NG, s));
  if ((rc = precondition(P, mlp, odd, 1, s))) return rc;
  k_fpcg_dir<<<stream_grid(m->NG, 1, 256, 8), 256, 0, s>>>(m->NG, v.r, v.dinv, v.z, v.p, st);
  BS_LAUNCH_CHECK();
  const int chunk = 8;
  const bool graph = flags & BS_CG_GRAPH;
  cudaGraphExec_t gexec = nullptr;
  auto capture = [&](bs_mlp *net) -> int {
    if (gexec) {
      cudaGraphExecDestroy(gexec);
      gexec = nullptr;
    }
    cudaStream_t cs = P->cap_stream;
    BS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int r2 = BS_OK;
    for (int c = 0; c < chunk && !r2; ++c) r2 = fpcg_iteration(P, net, odd, ff, x, cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (!r2 && e != cudaSuccess) r2 = fail(BS_ERR_CUDA, "fpcg capture: %s", cudaGetErrorString(e));
    if (!r2) {
      e = cudaGraphInstantiate(&gexec, g, 0);
      if (e != cudaSuccess) r2 = fail(BS_ERR_CUDA, "fpcg instantiate: %s", cudaGetErrorString(e));
    }
    if (g) cudaGraphDestroy(g);
    return r2;
  };
  if (graph && (rc = capture(mlp))) return rc;
  // Jacobi judges the learned correction: if the residual has not halved
  // within kStall iterations, the solve restarts from the current iterate
  // with the Jacobi preconditioner (z = D^-1 r, p = z) for good.  r.r is not
  // monotone in (F)CG: on these operators Jacobi-PCG itself has gone up to
  // about 7.5 N_G^(1/3) iterations without halving it, so the window is
  // 16 N_G^(1/3) (at least 1024) -- a guard against a correction that stalls
  // the solve, not a race against Jacobi.
  const int kStall = std::max(1024, (int)(16.0 * std::cbrt((double)m->NG)));
  bs_mlp *net = mlp;
  int switched_at = 0, window_iter = 0;
  double window_rr = INFINITY;
  for (int launched = 0; launched < maxit + chunk && !rc; launched += chunk) {
    if (graph) {
      if (cudaGraphLaunch(gexec, s) != cudaSuccess) rc = fail(BS_ERR_CUDA, "fpcg graph launch");
    } else {
      for (int c = 0; c < chunk && !rc; ++c) rc = fpcg_iteration(P, net, odd, ff, x, s);
    }
    if (rc) break;
    if (cudaMemcpyAsync(P->h_state, st, sizeof(CgState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = fail(BS_ERR_CUDA, "fpcg: state read back failed");
      break;
    }
    const CgState &h = *P->h_state;
    if (h.done) break;
    if (net && judge) {
      if (h.rr <= 0.25 * window_rr) {  // r.r down by 4: the residual has halved
        window_rr = h.rr;
        window_iter = h.iter;
      } else if (h.iter - window_iter >= kStall) {
        net = nullptr;
        switched_at = h.iter;
        if ((rc = precondition(P, nullptr, 0, 1, s))) break;
        k_fpcg_dir<<<stream_grid(m->NG, 1, 256, 8), 256, 0, s>>>(m->NG, v.r, v.dinv, v.z, v.p,
                                                               st);
        if (cudaGetLastError() != cudaSuccess) {
          rc = fail(BS_ERR_CUDA, "fpcg: restart launch failed");
          break;
        }
        if (graph && (rc = capture(nullptr))) break;
      }
    }
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  if (rc) return rc;
  BS_CUDA_TRY(cudaMemcpyAsync(P->h_state, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  BS_CUDA_TRY(cudaStreamSynchronize(s));
  const CgState &h = *P->h_state;
  if (h.done == 2)
    rc = fail(BS_ERR_BREAKDOWN, "bs_fpcg_learned: breakdown at iteration %d", h.iter);
  else if (!(h.rr <= h.eps))
    rc = fail(BS_ERR_NOT_CONVERGED, "bs_fpcg_learned: %d iterations", h.iter);
  if (info) {
    info->iterations = h.iter;
    info->fallbacks = h.nfallback;
    info->outer = switched_at;
    info->rr = h.rr;
    info->bb = h.bb;
    info->rel_residual = h.bb > 0 ? std::sqrt(h.rr / h.bb) : std::sqrt(h.rr);
    info->status = rc;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

}  // extern "C"
