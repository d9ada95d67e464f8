// bs_op.cuh -- the Helmholtz operator A = Z^T (c S_L + lambda M_L) Z of
// eqs. global_system, assembled_stiff, assembled_mass on affine cube
// elements with degree-N GLL bases (Sec. 2) and collocated quadrature.
//
// Per element, with K = D^T W D (the 1-D GLL stiffness, exact because the
// integrand has degree 2N-2), the stiffness is a sum of three one-directional
// contractions:
//   (S_e u)_ijk = (h/2) [ w_j w_k sum_m K_im u_mjk
//                       + w_i w_k sum_m K_jm u_imk
//                       + w_i w_j sum_m K_km u_ijm ],
// 3(N+1) fused multiply-adds per node, and the lumped mass is diagonal,
// (h/2)^3 w_i w_j w_k.  The kernel maps one thread to a column (i, j) of an
// element and walks k, keeping the column in registers; the element sits in
// shared memory.  Reading the input through the map (GATHER_IN) fuses the
// scatter Z p into the same pass, so the N_L-sized Z p is never stored.
//
// Fused form (FUSED): the map comes re-encoded (bs_map::d_ids_f) so that the
// kernel knows which global nodes have a single local copy -- element
// interiors and the faces on the natural boundary, 63% of the nodes at
// N = 7.  For those, Z^T is the identity: the kernel writes (A p)_g = +0 +
// (A_L Z p)_l straight into the global output and adds p_g (A p)_g to a
// per-block partial of p.Ap; only the shared nodes' local values go to the
// N_L buffer, for a gather over the shared rows alone.  The result is
// bitwise that of the unfused operator (a one-term row sum is +0 + v).
// Measured slower on GB300 (N = 7 on 48^3: 1.365 vs 1.244 ms per A p with
// the float-float kernel, 3.54 vs 3.44 ms in FP64): in the user's global
// numbering the single-copy nodes come in runs of N - 1 doubles and the
// shared rows between them, so both kernels write partial sectors of A p,
// which costs more than the N_L round trip saved.  Off by default.
#pragma once

#include "bs_gather.cuh"

namespace bs {

constexpr int kMaxNq = 16;  // degrees 1..15

// Per-problem constant tables, in device memory.
template <typename T>
struct OpTab {
  T K[kMaxNq * kMaxNq];  // K[i*Nq + m] = (D^T W D)_im
  T w[kMaxNq];           // GLL weights
};

template <int NQ>
struct OpShape {
  static constexpr int NQ2 = NQ * NQ;
  static constexpr int NP = NQ * NQ * NQ;
  static constexpr int EPB = NQ2 >= 128 ? 1 : 256 / NQ2;  // elements per block
  static constexpr int THREADS = ((EPB * NQ2 + 31) / 32) * 32;
};

// out = A_L in  on elements slot0 .. slot0 + EPB - 1 (slots index `order`
// when given, else elements directly), by a block of at least
// OpShape<NQ>::THREADS threads; every thread of the block must call it (it
// holds block barriers).  GATHER_IN: in is a global vector read through ids
// (masked nodes read as 0); else in is element-local.  g = h/2 (the
// c-independent stiffness factor), mlam = lambda (h/2)^3.  Elements visited
// in `order` (sorted by smallest global index) meet their neighbours' reads
// in L2.  s_u holds EPB * NQ^3 values, s_K NQ^2, s_w NQ.  FUSED (with
// GATHER_IN, ids the fused encoding): single-copy nodes go to outG, with
// p_g (A p)_g added to acc, shared ones to out; masked ones nowhere.
template <typename T, int NQ, bool GATHER_IN, bool FUSED = false>
__device__ __forceinline__ void ax_elements(int64_t slot0, int64_t E,
                                            const int32_t *__restrict__ order,
                                            const int32_t *__restrict__ ids,
                                            const T *__restrict__ in, T *__restrict__ out,
                                            const OpTab<T> *__restrict__ tab,
                                            const double *__restrict__ coef, T g, T mlam,
                                            T *s_u_all, T *s_K, T *s_w,
                                            T *__restrict__ outG = nullptr,
                                            Acc<T> *acc = nullptr) {
  static_assert(!FUSED || GATHER_IN, "the fused operator reads its input through the map");
  using S = OpShape<NQ>;
  __syncthreads();  // the shared buffers may still be in use by a previous call
  for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) s_K[t] = tab->K[(t / NQ) * NQ + t % NQ];
  for (int t = threadIdx.x; t < NQ; t += blockDim.x) s_w[t] = tab->w[t];
  const int le = threadIdx.x / S::NQ2;
  const int ij = threadIdx.x - le * S::NQ2;
  const int i = ij % NQ, j = ij / NQ;
  const int64_t slot = slot0 + le;
  const bool active = le < S::EPB && slot < E;
  const int64_t e = active && order ? (int64_t)order[slot] : slot;
  T *u = s_u_all + (le < S::EPB ? le : 0) * S::NP;
  T ureg[NQ];
  int32_t gid[FUSED ? NQ : 1];  // fused: the encoded id of each node of the column
  if (active) {
    const int64_t base = e * S::NP + ij;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      T v;
      if (FUSED) {
        const int32_t id = __ldcs(ids + base + k * S::NQ2);
        gid[k] = id;
        const int32_t gg = id >= 0 ? id : -2 - id;
        v = id != -1 ? in[gg] : T(0);
      } else if (GATHER_IN) {
        const int32_t id = __ldcs(ids + base + k * S::NQ2);
        v = id >= 0 ? in[id] : T(0);
      } else {
        v = __ldcs(in + base + k * S::NQ2);
      }
      ureg[k] = v;
      u[ij + k * S::NQ2] = v;
    }
  }
  __syncthreads();
  if (!active) return;
  const T c = coef ? T(coef[e]) : T(1);
  const T cg = c * g;
  const T wi = s_w[i], wj = s_w[j];
  const T wij = wi * wj;
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    T ar = T(0), as = T(0), at = T(0);
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      ar = fmaT(s_K[i * NQ + m], u[m + NQ * j + S::NQ2 * k], ar);
      as = fmaT(s_K[j * NQ + m], u[i + NQ * m + S::NQ2 * k], as);
      at = fmaT(s_K[k * NQ + m], ureg[m], at);
    }
    const T wk = s_w[k];
    T stiff = (wj * wk) * ar;
    stiff = fmaT(wi * wk, as, stiff);
    stiff = fmaT(wij, at, stiff);
    const T mass = mlam * (wij * wk) * ureg[k];
    const T res = fmaT(cg, stiff, mass);
    if (FUSED) {
      const int32_t id = gid[FUSED ? k : 0];
      if (id >= 0) {
        __stcs(out + e * S::NP + ij + k * S::NQ2, res);
      } else if (id != -1) {
        const T v = plus_zero(res);
        __stcs(outG + (-2 - id), v);
        acc->add(ureg[k], v);
      }
    } else {
      __stcs(out + e * S::NP + ij + k * S::NQ2, res);
    }
  }
}

template <typename T, int NQ, bool GATHER_IN, bool FUSED>
__global__ void __launch_bounds__(OpShape<NQ>::THREADS)
    k_ax_local(int64_t E, const int32_t *__restrict__ order, const int32_t *__restrict__ ids,
               const T *__restrict__ in, T *__restrict__ out, const OpTab<T> *__restrict__ tab,
               const double *__restrict__ coef, T g, T mlam, const CgState *st,
               T *__restrict__ outG, double *__restrict__ partials) {
  using S = OpShape<NQ>;
  __shared__ T s_u[S::EPB * S::NP];
  __shared__ T s_K[NQ * NQ];
  __shared__ T s_w[NQ];
  if (cg_halted(st)) return;
  Acc<T> acc;
  ax_elements<T, NQ, GATHER_IN, FUSED>((int64_t)blockIdx.x * S::EPB, E, order, ids, in, out,
                                       tab, coef, g, mlam, s_u, s_K, s_w, outG, &acc);
  if (FUSED && partials) {
    const double part = block_sum<S::THREADS>(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = part;
  }
}

// Blocks of the element kernels for E elements of degree N (the fused
// operator's partials hold one double per block).
inline int64_t ax_blocks(int N, int64_t E) {
  switch (N + 1) {
#define BS_AXB(NQ) \
  case NQ:         \
    return (E + OpShape<NQ>::EPB - 1) / OpShape<NQ>::EPB;
    BS_AXB(2) BS_AXB(3) BS_AXB(4) BS_AXB(5) BS_AXB(6) BS_AXB(7) BS_AXB(8) BS_AXB(9)
    BS_AXB(10) BS_AXB(11) BS_AXB(12) BS_AXB(13) BS_AXB(14) BS_AXB(15) BS_AXB(16)
#undef BS_AXB
    default:
      return 0;
  }
}

// FUSED: ids is the fused encoding, outG the global output, partials (or
// NULL: no dot product) ax_blocks(N, E) doubles.
template <typename T, bool GATHER_IN, bool FUSED = false>
int launch_ax_local(int N, int64_t E, const int32_t *order, const int32_t *ids, const T *in,
                    T *out,
                    const OpTab<T> *tab, const double *coef, T g, T mlam,
                    const CgState *st, cudaStream_t s, T *outG = nullptr,
                    double *partials = nullptr) {
  if (E == 0) return BS_OK;
#define BS_AX_CASE(NQ)                                                                   \
  case NQ: {                                                                             \
    using Sh = OpShape<NQ>;                                                              \
    const int64_t grid = (E + Sh::EPB - 1) / Sh::EPB;                                    \
    k_ax_local<T, NQ, GATHER_IN, FUSED><<<(unsigned)grid, Sh::THREADS, 0, s>>>(          \
        E, order, ids, in, out, tab, coef, g, mlam, st, outG, partials);                 \
    break;                                                                               \
  }
  switch (N + 1) {
    BS_AX_CASE(2)
    BS_AX_CASE(3)
    BS_AX_CASE(4)
    BS_AX_CASE(5)
    BS_AX_CASE(6)
    BS_AX_CASE(7)
    BS_AX_CASE(8)
    BS_AX_CASE(9)
    BS_AX_CASE(10)
    BS_AX_CASE(11)
    BS_AX_CASE(12)
    BS_AX_CASE(13)
    BS_AX_CASE(14)
    BS_AX_CASE(15)
    BS_AX_CASE(16)
    default:
      return fail(BS_ERR_ARG, "degree %d unsupported", N);
  }
#undef BS_AX_CASE
  BS_LAUNCH_CHECK();
  return BS_OK;
}

struct OpTabFF;  // bs_op_ff.cuh

}  // namespace bs

// A problem: the map, the geometry and the device scratch of the solvers.
struct bs_problem {
  int device;
  const bs_map *map;
  int32_t N;
  double h, lambda;
  double *d_coef;                 // [E] or NULL
  bs::OpTab<double> *d_tab;       // FP64 tables
  bs::OpTab<float> *d_tabf;       // FP32 tables
  bs::OpTabFF *d_tabff;           // float-pair tables of the float-float operator
  double *d_ApL;                  // [NL] local operator output (FP64 or FP32 view)
  double *d_vec;                  // 6 x [NG]: r, p, Ap, z, dinv, spare
  bs::CgState *d_state;
  double *d_partials;             // [kMaxPartials]
  double *d_op_partials;          // [ax_blocks(N, E)] the fused operator's block partials
  unsigned int *d_counter;
  bs::CgState *h_state;           // pinned host mirror for convergence checks
  cudaStream_t cap_stream;        // private stream for graph capture
  cudaGraphExec_t graph;          // cached CG chunk graph
  const void *graph_key[4];       // (x, variant, chunk, map) the graph was made for
  float *d_f32;                   // 4 x [NG + 8] FP32 vectors (refined solver), lazily
  double *d_Lvec;                 // 6 x [NL + 2 rounded up to even] scattered CG vectors, lazily
  uint8_t *d_owner;               // [NL + 16] 1 at the lowest local copy of each node, lazily
};
