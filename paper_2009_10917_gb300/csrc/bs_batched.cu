// bs_batched.cu -- many independent CG solves (Algorithm 1) of uneven size
// advanced together: one cooperative persistent launch per iteration for all
// solves that are still running, replayed as a CUDA graph.
//
// A launch runs the iteration in phases separated by grid barriers; each
// phase walks a work list of (solve, unit) items in grid-stride order:
//   A  fused scatter + element operator     items = (solve, element group)
//   B  gather with the p.Ap partial         items = (solve, gather tile)
//      -> the last tile of a solve to finish sums that solve's partials in
//         item order and forms alpha (deterministic, no float atomics)
//   C  fused update x += a p, r -= a Ap     items = (solve, 4096-entry chunk)
//      with the r.r partial; the last chunk forms beta and the stop flag
//   D  p = r + beta p                       items = (solve, chunk)
// The host reads one flag per solve at every convergence check and, once a
// quarter of the listed solves have stopped, rebuilds the work lists from the
// solves still running (and re-captures the graph), so finished solves stop
// costing even the check of their items.  The
// barrier spins are bounded (clock budget); on expiry the launch records
// BS_ERR_TIMEOUT and returns instead of waiting forever.
//
// The same kernel, instantiated for float, is the inner solver of the
// batched FP32-storage / FP64-refinement form: the outer FP64 residual
// b - A x and the update x = x + d run as ordinary launches over all solves.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "bs_op_ff.cuh"

namespace bs {

constexpr int kBBlock = 256;
constexpr int kBMaxNq = 9;                       // degrees 1..8 in a batch
constexpr int kBSmem = 2187;                     // max EPB * Nq^3 for Nq <= 9 (>= kTileNnz)
constexpr int kBChunk = 4096;                    // default vector entries per C/D item
constexpr long long kBarrierBudget = 1ll << 32;  // default clock cycles (~2 s) per barrier wait

// The barrier budget in force on this device (bs_set_wait_budget); read by
// every grid barrier, so a change also reaches launches replayed from graphs.
__device__ long long g_barrier_budget = kBarrierBudget;

struct BDesc {
  int NQ;
  int eo;      // 1: even-odd element operator for even NQ (bs_operator_mode at setup)
  int active;  // 1: participates in the current inner/outer step
  int64_t E, NG;
  int64_t NL, nnz, ntiles;  // bounds of the checked build's index tests
  const int32_t *ids, *order, *row_starts, *col_ids;
  const int2 *tiles;
  const double *coef;
  const OpTab<double> *tab;
  const OpTab<float> *tabf;
  const OpTabFF *tabff;
  double g, mlam;
  double *x, *r, *p, *Ap, *ApL;  // FP64 (x: the solution)
  const double *b;
  float *rf, *pf, *Apf, *df;     // FP32 inner vectors (refined form)
  float *ApLf;
  CgState *st;
  double bb, rr_true;            // outer (refined form)
  int outer, outer_done;
};

template <typename T> struct BV;
template <> struct BV<double> {
  static __device__ double *x(const BDesc &d) { return d.x; }
  static __device__ double *r(const BDesc &d) { return d.r; }
  static __device__ double *p(const BDesc &d) { return d.p; }
  static __device__ double *Ap(const BDesc &d) { return d.Ap; }
  static __device__ double *ApL(const BDesc &d) { return d.ApL; }
  static __device__ const OpTab<double> *tab(const BDesc &d) { return d.tab; }
  static __device__ double alpha(const CgState *s) { return s->alpha; }
  static __device__ double beta(const CgState *s) { return s->beta; }
};
template <> struct BV<float> {
  static __device__ float *x(const BDesc &d) { return d.df; }
  static __device__ float *r(const BDesc &d) { return d.rf; }
  static __device__ float *p(const BDesc &d) { return d.pf; }
  static __device__ float *Ap(const BDesc &d) { return d.Apf; }
  static __device__ float *ApL(const BDesc &d) { return d.ApLf; }
  static __device__ const OpTab<float> *tab(const BDesc &d) { return d.tabf; }
  static __device__ float alpha(const CgState *s) { return s->alpha_f; }
  static __device__ float beta(const CgState *s) { return s->beta_f; }
};

// Grid barrier for a cooperative launch: bar[0] counts arrivals, bar[1] is
// the generation.  Waits are bounded; returns false (all threads) if this or
// another block gave up, after recording BS_ERR_TIMEOUT in *err.
__device__ bool grid_sync(unsigned int *bar, int *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *vgen = bar + 1;
    const unsigned int gen = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long budget = *(volatile long long *)&g_barrier_budget;
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (clock64() - t0 > budget) {
          atomicExch(err, (int)BS_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok && *(volatile int *)err == 0;
  }
  __syncthreads();
  return s_ok;
}

__device__ __forceinline__ bool solve_off(const BDesc &d) {
  return !d.active || *(volatile const int *)&d.st->done != 0;
}

// The element operator as a real call: each degree keeps its own register
// allocation instead of the kernel taking the largest one of all degrees.
template <typename T, int NQ, bool GATHER_IN>
__device__ __noinline__ void ax_call(int64_t slot0, int64_t E, const int32_t *order,
                                     const int32_t *ids, const T *in, T *out,
                                     const OpTab<T> *tab, const double *coef, T g, T mlam,
                                     T *s_u, T *s_K, T *s_w) {
  ax_elements<T, NQ, GATHER_IN>(slot0, E, order, ids, in, out, tab, coef, g, mlam, s_u, s_K,
                                s_w);
}

// The FP64 even-odd element operator on elements [slot0, slot1): calls of
// EoShape<NQ, kBBlock>::EPB elements (the whole item: 256 / Nq^2 elements,
// every thread one (i, j) column).  The float-float and FP32 forms keep the
// direct element operator here: the even-odd group needs four times the
// direct form's shared memory (64 KB per block at Nq = 8), and with it the
// float-float batch (three blocks per SM) took 16.9 s instead of 15.7 s and
// the FP32 batch 16.4 s instead of 15.6 s, while the FP64 batch gained
// (28.6 s against 29.1 s).
template <int NQ>
__device__ __noinline__ void ax_call_eo(int64_t slot0, int64_t slot1, const int32_t *order,
                                        const int32_t *ids, const double *in, double *out,
                                        const OpTab<double> *tab, const double *coef, double g,
                                        double mlam, double *smem) {
  for (int64_t s0 = slot0; s0 < slot1; s0 += EoShape<NQ, kBBlock>::EPB)
    ax_elements_eo<double, NQ, true, false, kBBlock>(s0, slot1, order, ids, in, out, tab, coef,
                                                     g, mlam, smem, nullptr, nullptr);
}

// The float-float element operator (bs_op_ff.cuh) as a real call.
template <int NQ>
__device__ __noinline__ void ax_call_ff(int64_t slot0, int64_t E, const int32_t *order,
                                        const int32_t *ids, const double *in, double *out,
                                        const OpTabFF *tab, const double *coef, double g,
                                        double mlam, float *smem) {
  float *s_uh = smem, *s_ul = smem + kBSmem, *s_K = smem + 2 * kBSmem;
  float *s_w = s_K + 4 * kBMaxNq * kBMaxNq;
  ax_elements_ff<NQ, true>(slot0, E, order, ids, in, out, tab, coef, g, mlam, s_uh, s_ul, s_K,
                           s_w);
}

// Element operator on one item (block-uniform dispatch on the degree); FF:
// the float-float operator (FP64 form only).
template <typename T, bool GATHER_IN, bool FF = false>
__device__ void item_ax(const BDesc &d, int64_t slot0, const T *in, T *out, T *smem) {
  // elements of this item: [slot0, slot1)
  const int nq2 = d.NQ * d.NQ;
  const int64_t slot1 = slot0 + (nq2 >= 128 ? 1 : 256 / nq2) < d.E
                            ? slot0 + (nq2 >= 128 ? 1 : 256 / nq2)
                            : d.E;
  if constexpr (GATHER_IN && !FF && sizeof(T) == 8) {
    if (d.eo && (d.NQ == 2 || d.NQ == 4 || d.NQ == 6 || d.NQ == 8)) {
#define BS_EO_CASE(NQ)                                                                         \
  case NQ:                                                                                     \
    ax_call_eo<NQ>(slot0, slot1, d.order, d.ids, in, out, d.tab, d.coef, d.g, d.mlam, smem);   \
    return;
      switch (d.NQ) { BS_EO_CASE(2) BS_EO_CASE(4) BS_EO_CASE(6) BS_EO_CASE(8) default: return; }
#undef BS_EO_CASE
    }
  }
  if constexpr (FF) {
    static_assert(sizeof(T) == 8 && GATHER_IN, "float-float operator: FP64 form only");
    {
      float *fs = reinterpret_cast<float *>(smem);
#define BS_BF_CASE(NQ)                                                                        \
  case NQ:                                                                                    \
    ax_call_ff<NQ>(slot0, d.E, d.order, d.ids, (const double *)in, (double *)out, d.tabff,    \
                   d.coef, d.g, d.mlam, fs);                                                  \
    return;
      switch (d.NQ) {
        BS_BF_CASE(2)
        BS_BF_CASE(3)
        BS_BF_CASE(4)
        BS_BF_CASE(5)
        BS_BF_CASE(6)
        BS_BF_CASE(7)
        BS_BF_CASE(8)
        BS_BF_CASE(9)
        default:
          return;
      }
#undef BS_BF_CASE
    }
  } else {
  T *s_K = smem + kBSmem;
  T *s_w = s_K + kBMaxNq * kBMaxNq;
  const T g = (T)d.g, mlam = (T)d.mlam;
  const OpTab<T> *tab = BV<T>::tab(d);
#define BS_B_CASE(NQ)                                                                         \
  case NQ:                                                                                    \
    ax_call<T, NQ, GATHER_IN>(slot0, d.E, d.order, d.ids, in, out, tab, d.coef, g, mlam,      \
                              smem, s_K, s_w);                                                \
    break;
  switch (d.NQ) {
    BS_B_CASE(2)
    BS_B_CASE(3)
    BS_B_CASE(4)
    BS_B_CASE(5)
    BS_B_CASE(6)
    BS_B_CASE(7)
    BS_B_CASE(8)
    BS_B_CASE(9)
    default:
      break;
  }
#undef BS_B_CASE
  }
}

// Sum of part[a..b) in a fixed order over the block (valid in thread 0).
__device__ double sum_items(const double *part, int a, int b) {
  double v = 0.0;
  for (int i = a + (int)threadIdx.x; i < b; i += kBBlock) v = v + __ldcg(part + i);
  return block_sum<kBBlock>(v);
}

// Records this item's partial; returns true in the block that completes the
// solve's items, with *total = the sum over the solve's items in item order.
__device__ bool item_done(double part, double *parts, int item, int first, int last,
                          unsigned int *cnt, double *total) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    parts[item] = part;
    __threadfence();
    s_last = atomicAdd(cnt, 1u) == (unsigned int)(last - first - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  const double t = sum_items(parts, first, last);
  if (threadIdx.x == 0) {
    *total = t;
    *cnt = 0u;
  }
  return true;
}

struct BLists {
  const BDesc *d;
  int ns;                     // solves in d
  int chunk;                  // vector entries per C/D item
  const int2 *iA, *iB, *iC;
  int nA, nB, nC;
  const int4 *rng;            // [nsolves] (b0, b1, c0, c1): item ranges in lists B and C
  double *partB, *partC;
  unsigned int *cntB, *cntC;  // [nsolves] each
  unsigned int *bar;
  int *err;
  int *active;                // number of running solves
  int *sdone;                 // [nsolves] 0 while a solve's CG is running
  int *odone;                 // [nsolves] refined form: 0 while refinement continues
};

__device__ void stop_solve(const BLists &L, int s, CgState *st, int done) {
  st->done = done;
  L.sdone[s] = done;
  atomicSub(L.active, 1);
}

__device__ void finish_iteration(const BLists &L, int s, CgState *st, double rr_new) {
  const double beta = rr_new / st->rr;
  const int j = st->iter;
  st->beta = beta;
  st->beta_f = (float)beta;
  st->rr = rr_new;
  st->iter = j + 1;
  int done = 0;
  if (!isfinite(rr_new) || !isfinite(beta))
    done = 2;
  else if (rr_new <= st->eps)
    done = 1;
  else if (j + 1 >= st->maxit)
    done = 3;
  if (done) stop_solve(L, s, st, done);
}

// Shared memory of the element phase, in T: the element values, K and w
// (FP64 / FP32 operator), or, viewed as floats, the float pairs of the
// values, the four split tables and the split weights (float-float
// operator); in the FP64 form also the largest even-odd element group at
// this block width (Nq = 8: four elements of 4 x 512 values plus tables).
// Dynamic: 64 KB in the FP64 form, 19 KB float-float, 9 KB FP32.
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kBSmemDirect = kBSmem + 2 * kBMaxNq * kBMaxNq + 32;  // doubles
constexpr int kBSmemD =
    cmax(kBSmemDirect, cmax(cmax(EoShape<2, kBBlock>::SMEM, EoShape<4, kBBlock>::SMEM),
                            cmax(EoShape<6, kBBlock>::SMEM, EoShape<8, kBBlock>::SMEM)));
constexpr int kBSmemF = kBSmem + kBMaxNq * kBMaxNq + 16;  // floats
template <typename T, bool FF>
constexpr int iter_smem_bytes() {
  return sizeof(T) == 8 ? (FF ? kBSmemDirect * 8 : kBSmemD * 8) : kBSmemF * 4;
}
static int iter_smem(bool f32, bool ff) {
  return f32 ? iter_smem_bytes<float, false>()
             : (ff ? iter_smem_bytes<double, true>() : iter_smem_bytes<double, false>());
}

// One CG iteration of every running solve (cooperative launch).  U: vector
// entries per thread per sweep in the update phases (a tuning parameter);
// FF: the float-float element operator, which needs fewer registers, so
// that variant runs three blocks per SM instead of two.
template <typename T, int U, bool FF>
__global__ void __launch_bounds__(kBBlock, FF ? 3 : (sizeof(T) == 8 ? 2 : 4))
    k_batched_iter(BLists L) {
  extern __shared__ __align__(16) unsigned char bi_smem[];
  T *smem = reinterpret_cast<T *>(bi_smem);
  if (*(volatile int *)L.err) return;
  // A: ApL = A_L (Z p)
  for (int it = blockIdx.x; it < L.nA; it += gridDim.x) {
    const int2 w = L.iA[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    const BDesc &d = L.d[w.x];
    if (solve_off(d)) continue;
    item_ax<T, true, FF>(d, w.y, BV<T>::p(d), BV<T>::ApL(d), smem);
  }
  if (!grid_sync(L.bar, L.err)) return;
  // B: Ap = Z^T ApL; p.Ap -> alpha
  for (int it = blockIdx.x; it < L.nB; it += gridDim.x) {
    const int2 w = L.iB[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    const BDesc &d = L.d[w.x];
    if (solve_off(d)) continue;
    Acc<T> acc;
    __syncthreads();
    if (chk(w.y < d.ntiles, BS_CHK_BATCH))
      gather_tile<T, true, false>(d.tiles[w.y], d.tiles[w.y + 1], d.row_starts, d.col_ids,
                                  nullptr, BV<T>::ApL(d), BV<T>::Ap(d), BV<T>::p(d), smem, acc,
                                  GBounds{d.NG, d.nnz, d.NL, d.NG});
    const double part = block_sum<kBBlock>(acc.value());
    double pAp;
    const int4 rg = L.rng[w.x];
    if (item_done(part, L.partB, it, rg.x, rg.y, L.cntB + w.x, &pAp) && threadIdx.x == 0) {
      CgState *st = d.st;
      st->pAp = pAp;
      if (!(pAp > 0.0) || !isfinite(pAp)) {
        stop_solve(L, w.x, st, 2);
      } else {
        st->alpha = st->rr / pAp;
        st->alpha_f = (float)st->alpha;
      }
    }
  }
  if (!grid_sync(L.bar, L.err)) return;
  // C: x += alpha p; r -= alpha Ap; r.r -> beta, stop flag
  for (int it = blockIdx.x; it < L.nC; it += gridDim.x) {
    const int2 w = L.iC[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    const BDesc &d = L.d[w.x];
    if (solve_off(d)) continue;
    const T a = BV<T>::alpha(d.st), na = -a;
    T *x = BV<T>::x(d), *r = BV<T>::r(d);
    const T *p = BV<T>::p(d), *Ap = BV<T>::Ap(d);
    const int64_t i0 = (int64_t)w.y * L.chunk;
    const int64_t i1 = i0 + L.chunk < d.NG ? i0 + L.chunk : d.NG;
    Acc<T> acc;
    // U entries per thread per sweep, all 4 U loads issued together
    for (int64_t i = i0 + threadIdx.x; i < i1; i += U * kBBlock) {
      T pv[U], av[U], xv[U], rv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = i + u * kBBlock;
        const bool in = k < i1;
        pv[u] = in ? p[k] : T(0);
        av[u] = in ? Ap[k] : T(0);
        xv[u] = in ? x[k] : T(0);
        rv[u] = in ? r[k] : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = i + u * kBBlock;
        if (k < i1) {
          x[k] = fmaT(a, pv[u], xv[u]);
          const T ri = fmaT(na, av[u], rv[u]);
          r[k] = ri;
          acc.add(ri, ri);
        }
      }
    }
    const double part = block_sum<kBBlock>(acc.value());
    double rr;
    const int4 rg = L.rng[w.x];
    if (item_done(part, L.partC, it, rg.z, rg.w, L.cntC + w.x, &rr) && threadIdx.x == 0)
      finish_iteration(L, w.x, d.st, rr);
  }
  if (!grid_sync(L.bar, L.err)) return;
  // D: p = r + beta p
  for (int it = blockIdx.x; it < L.nC; it += gridDim.x) {
    const int2 w = L.iC[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    const BDesc &d = L.d[w.x];
    if (solve_off(d)) continue;
    const T bt = BV<T>::beta(d.st);
    T *p = BV<T>::p(d);
    const T *r = BV<T>::r(d);
    const int64_t i0 = (int64_t)w.y * L.chunk;
    const int64_t i1 = i0 + L.chunk < d.NG ? i0 + L.chunk : d.NG;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += U * kBBlock) {
      T rv[U], pv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = i + u * kBBlock;
        rv[u] = k < i1 ? r[k] : T(0);
        pv[u] = k < i1 ? p[k] : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = i + u * kBBlock;
        if (k < i1) p[k] = fmaT(T(1), rv[u], bt * pv[u]);
      }
    }
  }
}

// Start of a solve (FP64 form, x0 = 0): x = 0, r = p = b, r.r = b.b, stop rule.
__global__ void __launch_bounds__(kBBlock) k_batched_start(BLists L, double tol2, int maxit) {
  for (int it = blockIdx.x; it < L.nC; it += gridDim.x) {
    const int2 w = L.iC[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    const BDesc &d = L.d[w.x];
    const int64_t i0 = (int64_t)w.y * L.chunk;
    const int64_t i1 = i0 + L.chunk < d.NG ? i0 + L.chunk : d.NG;
    Acc<double> acc;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kBBlock) {
      const double bi = d.b[i];
      d.x[i] = 0.0;
      d.r[i] = bi;
      d.p[i] = bi;
      acc.add(bi, bi);
    }
    const double part = block_sum<kBBlock>(acc.value());
    double bb;
    const int4 rg = L.rng[w.x];
    if (item_done(part, L.partC, it, rg.z, rg.w, L.cntC + w.x, &bb) && threadIdx.x == 0) {
      CgState *st = d.st;
      st->bb = bb;
      st->rr = bb;
      st->eps = tol2 * bb;
      st->iter = 0;
      st->maxit = maxit;
      st->fixed = 0;
      st->hist = nullptr;
      st->done = !isfinite(bb) ? 2 : ((bb <= st->eps) ? 1 : (maxit <= 0 ? 3 : 0));
      L.sdone[w.x] = st->done;
      if (!st->done) atomicAdd(L.active, 1);
    }
  }
}

// Refined form, FP64 outer residual, phase 1: ApL = A_L (Z x) for solves
// that have not converged (x64 through the map, FP64 element operator).
__global__ void __launch_bounds__(kBBlock) k_batched_outer_ax(BLists L) {
  extern __shared__ __align__(16) unsigned char bo_smem[];  // iter_smem_bytes<double, false>()
  double *smem = reinterpret_cast<double *>(bo_smem);
  for (int it = blockIdx.x; it < L.nA; it += gridDim.x) {
    const int2 w = L.iA[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    const BDesc &d = L.d[w.x];
    if (d.outer_done) continue;
    item_ax<double, true>(d, w.y, d.x, d.ApL, smem);
  }
}

// phase 2: Ax = Z^T ApL (into Ap, FP64)
__global__ void __launch_bounds__(kBBlock) k_batched_outer_gather(BLists L) {
  __shared__ __align__(16) double smem[kTileNnz];
  for (int it = blockIdx.x; it < L.nB; it += gridDim.x) {
    const int2 w = L.iB[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    const BDesc &d = L.d[w.x];
    if (d.outer_done) continue;
    Acc<double> acc;
    __syncthreads();
    if (chk(w.y < d.ntiles, BS_CHK_BATCH))
      gather_tile<double, false, false>(d.tiles[w.y], d.tiles[w.y + 1], d.row_starts,
                                        d.col_ids, nullptr, d.ApL, d.Ap, nullptr, smem, acc,
                                        GBounds{d.NG, d.nnz, d.NL, d.NG});
  }
}

// phase 3: r = b - Ax (FP64), rf = (float) r, pf = rf, df = 0; the last item
// of a solve checks ||r|| <= tol ||b|| and, if not, starts its inner solve.
__global__ void __launch_bounds__(kBBlock)
    k_batched_outer_residual(BDesc *D, BLists L, double tol2, double itol2, int maxit,
                             int outer_maxit) {
  for (int it = blockIdx.x; it < L.nC; it += gridDim.x) {
    const int2 w = L.iC[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    BDesc &d = D[w.x];
    if (d.outer_done) continue;
    const int64_t i0 = (int64_t)w.y * L.chunk;
    const int64_t i1 = i0 + L.chunk < d.NG ? i0 + L.chunk : d.NG;
    Acc<double> acc;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kBBlock) {
      const double ri = d.b[i] - d.Ap[i];
      const float rfi = (float)ri;
      d.rf[i] = rfi;
      d.pf[i] = rfi;
      d.df[i] = 0.f;
      acc.add(ri, ri);
    }
    const double part = block_sum<kBBlock>(acc.value());
    double rr;
    const int4 rg = L.rng[w.x];
    if (item_done(part, L.partC, it, rg.z, rg.w, L.cntC + w.x, &rr) && threadIdx.x == 0) {
      CgState *st = d.st;
      d.rr_true = rr;
      if (!isfinite(rr)) {
        d.outer_done = 2;
      } else if (rr <= tol2 * d.bb) {
        d.outer_done = 1;
      } else if (d.outer >= outer_maxit || st->iter >= maxit) {
        d.outer_done = 3;
      }
      d.active = d.outer_done ? 0 : 1;
      L.odone[w.x] = d.outer_done;
      L.sdone[w.x] = d.active ? 0 : 1;
      if (d.active) {
        // the inner solve's r.r starts at (float) r . (float) r ~ rr
        st->rr = rr;
        st->bb = rr;
        st->eps = itol2 * rr;
        st->maxit = maxit;
        st->fixed = 0;
        st->hist = nullptr;
        st->done = 0;
        atomicAdd(L.active, 1);
      }
    }
  }
}

// x = x + (double) d for solves that ran an inner solve; count the step.
__global__ void __launch_bounds__(kBBlock) k_batched_outer_update(BDesc *D, BLists L) {
  for (int it = blockIdx.x; it < L.nC; it += gridDim.x) {
    const int2 w = L.iC[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    BDesc &d = D[w.x];
    if (!d.active) continue;
    const int64_t i0 = (int64_t)w.y * L.chunk;
    const int64_t i1 = i0 + L.chunk < d.NG ? i0 + L.chunk : d.NG;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kBBlock) d.x[i] = d.x[i] + (double)d.df[i];
    if (w.y == 0 && threadIdx.x == 0) d.outer += 1;
  }
}

// The inner FP32 iteration counts must accumulate across outer steps; the
// per-solve CgState keeps a running total in `iter` (never reset), and the
// stop rule compares it with maxit.
__global__ void k_batched_zero_x(BLists L) {
  for (int it = blockIdx.x; it < L.nC; it += gridDim.x) {
    const int2 w = L.iC[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    const BDesc &d = L.d[w.x];
    const int64_t i0 = (int64_t)w.y * L.chunk;
    const int64_t i1 = i0 + L.chunk < d.NG ? i0 + L.chunk : d.NG;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kBBlock) d.x[i] = 0.0;
  }
}

// b.b per solve and the initial outer state (refined form).
__global__ void __launch_bounds__(kBBlock) k_batched_bb(BDesc *D, BLists L) {
  for (int it = blockIdx.x; it < L.nC; it += gridDim.x) {
    const int2 w = L.iC[it];
    if (!chk(bs_pred_index(w.x, L.ns) && w.y >= 0, BS_CHK_BATCH)) continue;
    BDesc &d = D[w.x];
    const int64_t i0 = (int64_t)w.y * L.chunk;
    const int64_t i1 = i0 + L.chunk < d.NG ? i0 + L.chunk : d.NG;
    Acc<double> acc;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kBBlock) acc.add(d.b[i], d.b[i]);
    const double part = block_sum<kBBlock>(acc.value());
    double bb;
    const int4 rg = L.rng[w.x];
    if (item_done(part, L.partC, it, rg.z, rg.w, L.cntC + w.x, &bb) && threadIdx.x == 0) {
      d.bb = bb;
      d.outer = 0;
      d.outer_done = 0;
      d.st->iter = 0;
      d.st->done = 0;
    }
  }
}

// ------------------------------------------------------------ host side

struct Batch {
  int ns = 0;
  BDesc *d_desc = nullptr;
  int2 *d_items = nullptr;        // A, B and C lists, each at its full capacity
  int4 *d_rng = nullptr;
  double *d_parts = nullptr;
  unsigned int *d_cnt = nullptr;  // cntB[ns], cntC[ns], bar[2]
  int *d_flags = nullptr;         // err, active, sdone[ns], odone[ns]
  int *h_flags = nullptr;         // pinned mirror
  size_t capA = 0, capB = 0, capC = 0;
  std::vector<std::vector<int2>> hA, hB, hC;  // items of every solve
  std::vector<int> members;       // solves in the current lists
  BLists L{};
  int grid_iter = 0;
  int chunk = kBChunk, unroll = 4;  // tuning parameters (bs_batched_config)
  bool ff = false;                   // FP64 form with the float-float operator
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  ~Batch() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(d_desc);
    cudaFree(d_items);
    cudaFree(d_rng);
    cudaFree(d_parts);
    cudaFree(d_cnt);
    cudaFree(d_flags);
    if (h_flags) cudaFreeHost(h_flags);
  }
  int *h_sdone() { return h_flags + 2; }
  int *h_odone() { return h_flags + 2 + ns; }
};

// Work lists of the solves in `which` (ascending); every other solve gets
// empty item ranges.  Invalidates the captured graph.
static int upload_lists(Batch &B, const std::vector<int> &which, cudaStream_t s) {
  std::vector<int2> A, Bv, C;
  std::vector<int4> rng((size_t)B.ns, make_int4(0, 0, 0, 0));
  for (int sv : which) {
    A.insert(A.end(), B.hA[(size_t)sv].begin(), B.hA[(size_t)sv].end());
    int4 &r = rng[(size_t)sv];
    r.x = (int)Bv.size();
    Bv.insert(Bv.end(), B.hB[(size_t)sv].begin(), B.hB[(size_t)sv].end());
    r.y = (int)Bv.size();
    r.z = (int)C.size();
    C.insert(C.end(), B.hC[(size_t)sv].begin(), B.hC[(size_t)sv].end());
    r.w = (int)C.size();
  }
  int2 *dA = B.d_items, *dB = B.d_items + B.capA, *dC = B.d_items + B.capA + B.capB;
  if (!A.empty())
    BS_CUDA_TRY(cudaMemcpyAsync(dA, A.data(), sizeof(int2) * A.size(), cudaMemcpyHostToDevice, s));
  if (!Bv.empty())
    BS_CUDA_TRY(
        cudaMemcpyAsync(dB, Bv.data(), sizeof(int2) * Bv.size(), cudaMemcpyHostToDevice, s));
  if (!C.empty())
    BS_CUDA_TRY(cudaMemcpyAsync(dC, C.data(), sizeof(int2) * C.size(), cudaMemcpyHostToDevice, s));
  BS_CUDA_TRY(cudaMemcpyAsync(B.d_rng, rng.data(), sizeof(int4) * B.ns, cudaMemcpyHostToDevice, s));
  BS_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
  B.L.nA = (int)A.size();
  B.L.nB = (int)Bv.size();
  B.L.nC = (int)C.size();
  B.members = which;
  if (B.graph) {
    cudaGraphExecDestroy(B.graph);
    B.graph = nullptr;
  }
  return BS_OK;
}

// Reads err, active and the per-solve flags back to the host.
static int read_flags(Batch &B, cudaStream_t s) {
  BS_CUDA_TRY(cudaMemcpyAsync(B.h_flags, B.d_flags, sizeof(int) * (2 + 2 * (size_t)B.ns),
                              cudaMemcpyDeviceToHost, s));
  BS_CUDA_TRY(cudaStreamSynchronize(s));
  return BS_OK;
}

static int build_batch(Batch &B, int ns, const bs_problem *const *P, const double *const *b,
                       double *const *x, bool f32) {
  B.ns = ns;
  std::vector<BDesc> desc((size_t)ns);
  B.hA.assign((size_t)ns, {});
  B.hB.assign((size_t)ns, {});
  B.hC.assign((size_t)ns, {});
  for (int s = 0; s < ns; ++s) {
    const bs_problem *p = P[s];
    const bs_map *m = p->map;
    BDesc &d = desc[(size_t)s];
    memset(&d, 0, sizeof(d));
    d.NQ = p->N + 1;
    d.eo = g_op_evenodd;
    d.active = 1;
    d.E = m->E;
    d.NG = m->NG;
    d.NL = m->NL;
    d.nnz = m->nnz;
    d.ntiles = m->ntiles;
    d.ids = m->d_ids;
    d.order = m->d_elem_order;
    d.row_starts = m->d_row_starts;
    d.col_ids = m->d_col_ids;
    d.tiles = m->d_tiles;
    d.coef = p->d_coef;
    d.tab = p->d_tab;
    d.tabf = p->d_tabf;
    d.tabff = p->d_tabff;
    d.g = 0.5 * p->h;
    d.mlam = p->lambda * d.g * d.g * d.g;
    const int64_t sv = m->NG + 2;
    d.x = x[s];
    d.b = b[s];
    d.r = p->d_vec;
    d.p = p->d_vec + sv;
    d.Ap = p->d_vec + 2 * sv;
    d.ApL = p->d_ApL;
    if (f32) {
      const size_t n = (size_t)m->NG + 8;
      d.rf = p->d_f32;
      d.pf = p->d_f32 + n;
      d.Apf = p->d_f32 + 2 * n;
      d.df = p->d_f32 + 3 * n;
      d.ApLf = reinterpret_cast<float *>(p->d_ApL);
    }
    d.st = p->d_state;
    const int nq2 = d.NQ * d.NQ;
    const int epb = nq2 >= 128 ? 1 : 256 / nq2;
    for (int64_t e = 0; e < m->E; e += epb) B.hA[(size_t)s].push_back(make_int2(s, (int)e));
    for (int64_t t = 0; t < m->ntiles; ++t) B.hB[(size_t)s].push_back(make_int2(s, (int)t));
    const int64_t nch = (m->NG + B.chunk - 1) / B.chunk;
    for (int64_t c = 0; c < (nch > 0 ? nch : 1); ++c)
      B.hC[(size_t)s].push_back(make_int2(s, (int)c));
    B.capA += B.hA[(size_t)s].size();
    B.capB += B.hB[(size_t)s].size();
    B.capC += B.hC[(size_t)s].size();
  }
  BS_CUDA_TRY(cudaMalloc(&B.d_desc, sizeof(BDesc) * ns));
  BS_CUDA_TRY(cudaMemcpy(B.d_desc, desc.data(), sizeof(BDesc) * ns, cudaMemcpyHostToDevice));
  BS_CUDA_TRY(cudaMalloc(&B.d_items, sizeof(int2) * (B.capA + B.capB + B.capC)));
  BS_CUDA_TRY(cudaMalloc(&B.d_rng, sizeof(int4) * ns));
  BS_CUDA_TRY(cudaMalloc(&B.d_parts, sizeof(double) * (B.capB + B.capC)));
  BS_CUDA_TRY(cudaMalloc(&B.d_cnt, sizeof(unsigned int) * (2 * ns + 2)));
  BS_CUDA_TRY(cudaMemset(B.d_cnt, 0, sizeof(unsigned int) * (2 * ns + 2)));
  BS_CUDA_TRY(cudaMalloc(&B.d_flags, sizeof(int) * (2 + 2 * (size_t)ns)));
  BS_CUDA_TRY(cudaMemset(B.d_flags, 0, sizeof(int) * (2 + 2 * (size_t)ns)));
  BS_CUDA_TRY(cudaMallocHost(&B.h_flags, sizeof(int) * (2 + 2 * (size_t)ns)));
  BS_CUDA_TRY(cudaStreamCreateWithFlags(&B.cap, cudaStreamNonBlocking));
  BLists &L = B.L;
  L.d = B.d_desc;
  L.ns = ns;
  L.chunk = B.chunk;
  L.iA = B.d_items;
  L.iB = B.d_items + B.capA;
  L.iC = B.d_items + B.capA + B.capB;
  L.rng = B.d_rng;
  L.partB = B.d_parts;
  L.partC = B.d_parts + B.capB;
  L.cntB = B.d_cnt;
  L.cntC = B.d_cnt + ns;
  L.bar = B.d_cnt + 2 * ns;
  L.err = B.d_flags;
  L.active = B.d_flags + 1;
  L.sdone = B.d_flags + 2;
  L.odone = B.d_flags + 2 + ns;
  std::vector<int> all((size_t)ns);
  for (int i = 0; i < ns; ++i) all[(size_t)i] = i;
  return upload_lists(B, all, nullptr);
}

template <typename T, bool FF>
static void *iter_kernel_ff(int unroll) {
  switch (unroll) {
    case 1: return (void *)k_batched_iter<T, 1, FF>;
    case 2: return (void *)k_batched_iter<T, 2, FF>;
    case 8: return (void *)k_batched_iter<T, 8, FF>;
    default: return (void *)k_batched_iter<T, 4, FF>;
  }
}

template <typename T>
static void *iter_kernel(int unroll, bool ff = false) {
  if constexpr (sizeof(T) == 8) {
    if (ff) return iter_kernel_ff<double, true>(unroll);
  }
  return iter_kernel_ff<T, false>(unroll);
}

template <typename T>
static int launch_iter(Batch &B, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)B.grid_iter);
  cfg.blockDim = dim3(kBBlock);
  const int smem = iter_smem(sizeof(T) == 4, B.ff);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void *args[] = {&B.L};
  const void *kern = iter_kernel<T>(B.unroll, B.ff);
  if (occupancy_blocks_smem(kern, kBBlock, smem) < 1)  // sets the smem limit
    return fail(BS_ERR_CUDA, "batched CG: shared memory refused");
  BS_CUDA_TRY(cudaLaunchKernelExC(&cfg, kern, args));
  return BS_OK;
}

// Run iterations in chunks (optionally one graph per chunk) until no solve
// is running or a device error is recorded; drop stopped solves from the
// lists as they accumulate.
template <typename T>
static int iterate(Batch &B, bool graph, int maxit, cudaStream_t s) {
  const int chunk = 8;
  for (int launched = 0; launched < maxit + chunk; launched += chunk) {
    if (graph && !B.graph) {
      BS_CUDA_TRY(cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal));
      int rc = BS_OK;
      for (int c = 0; c < chunk && rc == BS_OK; ++c) rc = launch_iter<T>(B, B.cap);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(B.cap, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return fail(BS_ERR_CUDA, "batched capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&B.graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        B.graph = nullptr;
        return fail(BS_ERR_CUDA, "batched instantiate: %s", cudaGetErrorString(e));
      }
    }
    if (graph) {
      BS_CUDA_TRY(cudaGraphLaunch(B.graph, s));
    } else {
      for (int c = 0; c < chunk; ++c)
        if (int rc = launch_iter<T>(B, s)) return rc;
    }
    if (int rc = read_flags(B, s)) return rc;
    if (B.h_flags[0]) return fail(B.h_flags[0], "batched CG: device barrier timed out");
    const int running = B.h_flags[1];
    if (running <= 0) break;
    if (4 * running <= 3 * (int)B.members.size()) {
      std::vector<int> still;
      for (int m : B.members)
        if (B.h_sdone()[m] == 0) still.push_back(m);
      if (int rc = upload_lists(B, still, s)) return rc;
    }
  }
  return BS_OK;
}

// Cooperative grid: SMs x blocks per SM, the occupancy maximum or fewer
// (want > 0), at `smem` bytes of dynamic shared memory per block.
static int occupancy_grid(const void *kern, int smem, int want = 0) {
  DeviceInfo di;
  if (device_info(&di)) return 0;
  int bps = occupancy_blocks_smem(kern, kBBlock, smem);
  if (bps < 1) return 0;
  if (want > 0 && want < bps) bps = want;
  return bps * di.sms;
}

}  // namespace bs

namespace bs {

// Validates the arguments and prepares the FP32 scratch of the refined form.
static int check_batch(int32_t nsolves, const bs_problem *const *probs, const double *const *b,
                       double *const *x, double tol, int32_t maxit, int32_t flags,
                       const bs_batched_config *cfg, const char *fn) {
  BS_ARG(nsolves >= 1 && probs && b, "%s: empty or NULL arguments", fn);
  BS_ARG(maxit >= 0, "%s: maxit < 0", fn);
  BS_ARG(tol >= 0.0 && std::isfinite(tol), "%s: bad tol", fn);
  BS_ARG(!(flags & ~(BS_CG_GRAPH | BS_CG_REFINED_F32 | BS_CG_FF_OPERATOR)),
         "%s: only BS_CG_GRAPH, BS_CG_REFINED_F32 and BS_CG_FF_OPERATOR are supported", fn);
  BS_ARG(!((flags & BS_CG_REFINED_F32) && (flags & BS_CG_FF_OPERATOR)),
         "%s: BS_CG_FF_OPERATOR applies to the FP64 form only", fn);
  if (cfg) {
    const int c = cfg->chunk, u = cfg->unroll;
    BS_ARG(c == 0 || (c >= 1024 && c <= 65536 && (c & (c - 1)) == 0),
           "%s: chunk %d is not 0 or a power of two in [1024, 65536]", fn, c);
    BS_ARG(u == 0 || u == 1 || u == 2 || u == 4 || u == 8, "%s: unroll %d not in {1,2,4,8}", fn,
           u);
    BS_ARG(cfg->blocks_per_sm >= 0, "%s: blocks_per_sm < 0", fn);
  }
  const bool f32 = flags & BS_CG_REFINED_F32;
  int dev = -1;
  BS_CUDA_TRY(cudaGetDevice(&dev));
  for (int s = 0; s < nsolves; ++s) {
    BS_ARG(probs[s] && b[s] && (!x || x[s]), "%s: NULL entry %d", fn, s);
    BS_ARG(probs[s]->device == dev, "%s: problem %d on another device", fn, s);
    BS_ARG(probs[s]->N + 1 <= kBMaxNq, "%s: problem %d has degree %d > %d", fn, s, probs[s]->N,
           kBMaxNq - 1);
    BS_ARG(probs[s]->map->NG > 0, "%s: problem %d is empty", fn, s);
    BS_ARG(!probs[s]->d_geo, "%s: problem %d has geometric factors (not batched)", fn, s);
    for (int t = 0; t < s; ++t) BS_ARG(probs[t] != probs[s], "%s: problem %d repeats %d", fn, s, t);
    if (f32 && !probs[s]->d_f32) {
      bs_problem *p = const_cast<bs_problem *>(probs[s]);
      BS_CUDA_TRY(cudaMalloc(&p->d_f32, sizeof(float) * 4 * ((size_t)p->map->NG + 8)));
    }
  }
  return BS_OK;
}

// Sets up a batch with the given configuration (chunk, unroll, grid).
static int setup_batch(Batch &B, int32_t nsolves, const bs_problem *const *probs,
                       const double *const *b, double *const *x, int32_t flags,
                       const bs_batched_config *cfg) {
  const bool f32 = flags & BS_CG_REFINED_F32;
  if (cfg && cfg->chunk) B.chunk = cfg->chunk;
  if (cfg && cfg->unroll) B.unroll = cfg->unroll;
  B.ff = flags & BS_CG_FF_OPERATOR;
  if (int rc = build_batch(B, nsolves, probs, b, x, f32)) return rc;
  B.grid_iter = occupancy_grid(f32 ? iter_kernel<float>(B.unroll)
                                   : iter_kernel<double>(B.unroll, B.ff),
                               iter_smem(f32, B.ff),
                               cfg ? cfg->blocks_per_sm : 0);
  if (B.grid_iter < 1) return fail(BS_ERR_CUDA, "batched CG: no cooperative grid");
  return BS_OK;
}

static int solve_batched(int32_t nsolves, const bs_problem *const *probs, const double *const *b,
                         double *const *x, double tol, int32_t maxit, int32_t flags,
                         const bs_batched_config *cfg, bs_cg_info *infos, void *stream) {
  const auto t0 = std::chrono::steady_clock::now();
  BS_ARG(x != nullptr, "bs_cg_solve_batched: x is NULL");
  if (int rc = check_batch(nsolves, probs, b, x, tol, maxit, flags, cfg, "bs_cg_solve_batched"))
    return rc;
  const bool f32 = flags & BS_CG_REFINED_F32;
  cudaStream_t s = as_stream(stream);
  Batch B;
  int rc = setup_batch(B, nsolves, probs, b, x, flags, cfg);
  if (rc) return rc;
  const bool graph = flags & BS_CG_GRAPH;
  const int G = stream_grid((int64_t)B.capC, 1, 1, 8);
  const int GA =
      occupancy_grid((const void *)k_batched_outer_ax, iter_smem_bytes<double, false>());
  if (GA < 1) return fail(BS_ERR_CUDA, "batched CG: no grid for the outer residual");
  if (!f32) {
    k_batched_start<<<G, kBBlock, 0, s>>>(B.L, tol * tol, maxit);
    BS_LAUNCH_CHECK();
    rc = iterate<double>(B, graph, maxit, s);
  } else {
    const double itol = 1e-4;
    const int outer_maxit = 50;
    k_batched_zero_x<<<G, kBBlock, 0, s>>>(B.L);
    k_batched_bb<<<G, kBBlock, 0, s>>>(B.d_desc, B.L);
    BS_LAUNCH_CHECK();
    for (int step = 0; step <= outer_maxit && rc == BS_OK; ++step) {
      // solves whose refinement continues
      if (step > 0) {
        if ((rc = read_flags(B, s))) break;
        std::vector<int> open;
        for (int i = 0; i < nsolves; ++i)
          if (B.h_odone()[i] == 0) open.push_back(i);
        if (open.empty()) break;
        if ((rc = upload_lists(B, open, s))) break;
      }
      BS_CUDA_TRY(cudaMemsetAsync(B.L.active, 0, sizeof(int), s));
      k_batched_outer_ax<<<GA, kBBlock, iter_smem_bytes<double, false>(), s>>>(B.L);
      k_batched_outer_gather<<<G, kBBlock, 0, s>>>(B.L);
      k_batched_outer_residual<<<G, kBBlock, 0, s>>>(B.d_desc, B.L, tol * tol, itol * itol,
                                                      maxit, outer_maxit);
      BS_LAUNCH_CHECK();
      if ((rc = read_flags(B, s))) break;
      if (B.h_flags[1] <= 0) break;  // every solve has converged or stopped
      std::vector<int> inner;
      for (int m : B.members)
        if (B.h_sdone()[m] == 0) inner.push_back(m);
      if ((rc = upload_lists(B, inner, s))) break;
      rc = iterate<float>(B, graph, maxit, s);
      if (rc) break;
      if ((rc = upload_lists(B, inner, s))) break;  // x += d for this step's solves
      k_batched_outer_update<<<G, kBBlock, 0, s>>>(B.d_desc, B.L);
      BS_LAUNCH_CHECK();
    }
  }
  // results
  std::vector<BDesc> desc((size_t)nsolves);
  std::vector<CgState> st((size_t)nsolves);
  BS_CUDA_TRY(cudaStreamSynchronize(s));
  BS_CUDA_TRY(cudaMemcpy(desc.data(), B.d_desc, sizeof(BDesc) * nsolves, cudaMemcpyDeviceToHost));
  for (int i = 0; i < nsolves; ++i)
    BS_CUDA_TRY(cudaMemcpy(&st[(size_t)i], probs[i]->d_state, sizeof(CgState),
                           cudaMemcpyDeviceToHost));
  const double secs =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = rc;
  for (int i = 0; i < nsolves; ++i) {
    const CgState &h = st[(size_t)i];
    int status = BS_OK;
    double rel;
    if (!f32) {
      if (h.done == 2) status = BS_ERR_BREAKDOWN;
      else if (!(h.rr <= h.eps)) status = BS_ERR_NOT_CONVERGED;
      rel = h.bb > 0 ? std::sqrt(h.rr / h.bb) : std::sqrt(h.rr);
    } else {
      const BDesc &d = desc[(size_t)i];
      if (d.outer_done == 2 || h.done == 2) status = BS_ERR_BREAKDOWN;
      else if (d.outer_done != 1) status = BS_ERR_NOT_CONVERGED;
      rel = d.bb > 0 ? std::sqrt(d.rr_true / d.bb) : std::sqrt(d.rr_true);
    }
    if (rc) status = rc;
    if (!worst && status) worst = status;
    if (infos) {
      bs_cg_info &o = infos[i];
      memset(&o, 0, sizeof(o));
      o.iterations = h.iter;
      o.status = status;
      o.outer = f32 ? desc[(size_t)i].outer : 0;
      o.rr = f32 ? desc[(size_t)i].rr_true : h.rr;
      o.bb = f32 ? desc[(size_t)i].bb : h.bb;
      o.rel_residual = rel;
      o.seconds = secs;
    }
  }
  if (worst && !rc) return fail(worst, "bs_cg_solve_batched: some solves did not converge");
  return rc;
}

// Candidates: chunk x unroll x blocks per SM; each runs `iters` iterations
// (after one untimed) of the real solves from x = 0 into scratch solution
// vectors, timed with CUDA events; the fastest wins.
static int autotune(int32_t nsolves, const bs_problem *const *probs, const double *const *b,
                    int32_t flags, int32_t iters, bs_batched_config *best, double *best_ms,
                    void *stream) {
  if (int rc = check_batch(nsolves, probs, b, nullptr, 0.0, 1 << 30, flags, nullptr,
                           "bs_cg_batched_autotune"))
    return rc;
  BS_ARG(best != nullptr && iters >= 1, "bs_cg_batched_autotune: NULL best or iters < 1");
  const bool f32 = flags & BS_CG_REFINED_F32;
  cudaStream_t s = as_stream(stream);
  std::vector<double *> xs((size_t)nsolves, nullptr);
  int rc = BS_OK;
  for (int i = 0; i < nsolves && !rc; ++i)
    if (cudaMalloc(&xs[(size_t)i], sizeof(double) * (size_t)probs[i]->map->NG) != cudaSuccess)
      rc = fail(BS_ERR_ALLOC, "bs_cg_batched_autotune: scratch solution %d", i);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = fail(BS_ERR_CUDA, "bs_cg_batched_autotune: events");
  double bestv = INFINITY;
  const int chunks[] = {2048, 4096, 8192, 16384};
  const int unrolls[] = {2, 4, 8};
  const int bpss[] = {1, 0};
  for (int c : chunks)
    for (int u : unrolls)
      for (int bp : bpss) {
        if (rc) break;
        bs_batched_config cfg{c, bp, u};
        Batch B;
        if ((rc = setup_batch(B, nsolves, probs, b, xs.data(), flags, &cfg))) break;
        const int G = stream_grid((int64_t)B.capC, 1, 1, 8);
        if (!f32) {
          k_batched_start<<<G, kBBlock, 0, s>>>(B.L, 0.0, 1 << 30);
        } else {
          // the first inner solve of the refined form: r = b (x = 0)
          k_batched_zero_x<<<G, kBBlock, 0, s>>>(B.L);
          k_batched_bb<<<G, kBBlock, 0, s>>>(B.d_desc, B.L);
          const int GA =
              occupancy_grid((const void *)k_batched_outer_ax, iter_smem_bytes<double, false>());
          if (GA < 1) {
            rc = fail(BS_ERR_CUDA, "bs_cg_batched_autotune: no grid for the outer residual");
            break;
          }
          k_batched_outer_ax<<<GA, kBBlock, iter_smem_bytes<double, false>(), s>>>(B.L);
          k_batched_outer_gather<<<G, kBBlock, 0, s>>>(B.L);
          k_batched_outer_residual<<<G, kBBlock, 0, s>>>(B.d_desc, B.L, 0.0, 0.0, 1 << 30, 50);
        }
        if (cudaGetLastError() != cudaSuccess) {
          rc = fail(BS_ERR_CUDA, "bs_cg_batched_autotune: start launch");
          break;
        }
        rc = f32 ? launch_iter<float>(B, s) : launch_iter<double>(B, s);
        if (!rc) BS_CUDA_TRY(cudaEventRecord(e0, s));
        for (int k = 0; k < iters && !rc; ++k)
          rc = f32 ? launch_iter<float>(B, s) : launch_iter<double>(B, s);
        if (rc) break;
        BS_CUDA_TRY(cudaEventRecord(e1, s));
        BS_CUDA_TRY(cudaEventSynchronize(e1));
        if ((rc = read_flags(B, s))) break;
        if (B.h_flags[0]) {
          rc = fail(B.h_flags[0], "bs_cg_batched_autotune: device barrier timed out");
          break;
        }
        float ms = 0.f;
        BS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        const double per = ms / iters;
        if (per < bestv) {
          bestv = per;
          *best = cfg;
        }
      }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  for (double *p : xs) cudaFree(p);
  if (!rc && best_ms) *best_ms = bestv;
  return rc;
}

}  // namespace bs

using namespace bs;

extern "C" {

int bs_cg_solve_batched(int32_t nsolves, const bs_problem *const *probs, const double *const *b,
                        double *const *x, double tol, int32_t maxit, int32_t flags,
                        bs_cg_info *infos, void *stream) {
  return solve_batched(nsolves, probs, b, x, tol, maxit, flags, nullptr, infos, stream);
}

int bs_cg_solve_batched_ex(int32_t nsolves, const bs_problem *const *probs,
                           const double *const *b, double *const *x, double tol, int32_t maxit,
                           int32_t flags, const bs_batched_config *cfg, bs_cg_info *infos,
                           void *stream) {
  return solve_batched(nsolves, probs, b, x, tol, maxit, flags, cfg, infos, stream);
}

int bs_set_wait_budget(int64_t cycles, int64_t *previous) {
  long long prev = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&prev, g_barrier_budget, sizeof(prev));
  if (e != cudaSuccess)
    return fail(BS_ERR_CUDA, "bs_set_wait_budget: read: %s", cudaGetErrorString(e));
  const long long v = cycles > 0 ? (long long)cycles : kBarrierBudget;
  e = cudaMemcpyToSymbol(g_barrier_budget, &v, sizeof(v));
  if (e != cudaSuccess)
    return fail(BS_ERR_CUDA, "bs_set_wait_budget: write: %s", cudaGetErrorString(e));
  if (previous) *previous = prev;
  return BS_OK;
}

int bs_cg_batched_autotune(int32_t nsolves, const bs_problem *const *probs,
                           const double *const *b, int32_t flags, int32_t iters,
                           bs_batched_config *best, double *ms_per_iteration, void *stream) {
  return autotune(nsolves, probs, b, flags, iters, best, ms_per_iteration, stream);
}

}  // extern "C"
