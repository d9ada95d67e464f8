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
  T D[kMaxNq * kMaxNq];  // D[a*Nq + i] = l_i'(r_a), the GLL derivative matrix
  T w[kMaxNq];           // GLL weights
  // Even-odd halves of Kh = W^-1 K (centrosymmetric; even Nq only), h = Nq/2:
  // Ee[a*h + m] = (Kh_am + Kh_a,Nq-1-m) / 2, Eo[a*h + m] = (Kh_am - Kh_a,Nq-1-m) / 2.
  T Ee[(kMaxNq / 2) * (kMaxNq / 2)];
  T Eo[(kMaxNq / 2) * (kMaxNq / 2)];
  int64_t ne, ng;  // the problem's E and N_G (index checks of the checked build)
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
  bool active = le < S::EPB && slot < E;
  const int64_t e = active && order ? (int64_t)order[slot] : slot;
  if (active && !chk(bs_pred_index(e, tab->ne), BS_CHK_OP_ENTRY)) active = false;
  T *u = s_u_all + (le < S::EPB ? le : 0) * S::NP;
  T ureg[NQ];
  int32_t gid[FUSED ? NQ : 1];  // fused: the encoded id of each node of the column
  if (active) {
    const int64_t base = e * S::NP + ij;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      T v;
      if (FUSED) {
        int32_t id = __ldcs(ids + base + k * S::NQ2);
        if (!chk(bs_pred_fused_entry(id, tab->ng), BS_CHK_OP_ENTRY)) id = -1;
        gid[k] = id;
        const int32_t gg = id >= 0 ? id : -2 - id;
        v = id != -1 ? in[gg] : T(0);
      } else if (GATHER_IN) {
        int32_t id = __ldcs(ids + base + k * S::NQ2);
        if (!chk(bs_pred_map_entry(id, tab->ng), BS_CHK_OP_ENTRY)) id = -1;
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

// ---------------------------------------------------------------- even-odd form
//
// The GLL nodes are symmetric about 0, so Kh = W^-1 K (K = D^T W D) is
// centrosymmetric: Kh_{N-a, N-m} = Kh_{a m}.  With e_m = u_m + u_{N-m} and
// o_m = u_m - u_{N-m} (m < h = Nq/2; Solomonoff's even-odd decomposition of a
// spectral differentiation matrix), one pair of outputs of a 1-D contraction
// costs two half-length sums,
//   (Kh u)_a = sum_m Ee_am e_m + sum_m Eo_am o_m,
//   (Kh u)_{N-a} = sum_m Ee_am e_m - sum_m Eo_am o_m,
// and, because stiffness and mass both carry w_i w_j w_k,
//   (A_L u)_ijk = w_i w_j w_k (c (h/2) [(Kh u)_r + (Kh u)_s + (Kh u)_t] + lambda (h/2)^3 u_ijk).
// About 24 FP64 operations per node instead of 32 (the element kernel is
// FP64-pipe bound on GB300).  Even Nq only, up to 10.  Per element: the
// column pairs along r and along s get their e/o values computed once into
// shared memory; then each thread contracts one output pair along r (threads
// with i < h) or along s (the others), and, from its own column in registers,
// all outputs along t; a last pass sums the three per node.  BT: the block
// width the element group is sized for (128 for the element kernels; the
// batched kernel's 256-thread blocks take twice the elements per call).
template <int NQ, int BT = 128>
struct EoShape {
  static constexpr int H = NQ / 2;
  static constexpr int NQ2 = NQ * NQ;
  static constexpr int NP = NQ * NQ2;
  static constexpr int EPB = NQ2 >= BT ? 1 : BT / NQ2;  // elements per block
  static constexpr int THREADS = ((EPB * NQ2 + 31) / 32) * 32;
  static constexpr int SMEM = EPB * 4 * NP + 2 * H * H + NQ;  // values of T
};
template <int NQ>
constexpr bool use_eo() {
  return NQ % 2 == 0 && NQ <= 10;
}

// As ax_elements (same arguments, FUSED likewise), by a block of at least
// EoShape<NQ, BT>::THREADS threads; smem holds EoShape<NQ, BT>::SMEM values.
template <typename T, int NQ, bool GATHER_IN, bool FUSED, int BT = 128>
__device__ __forceinline__ void ax_elements_eo(int64_t slot0, int64_t E,
                                               const int32_t *__restrict__ order,
                                               const int32_t *__restrict__ ids,
                                               const T *__restrict__ in, T *__restrict__ out,
                                               const OpTab<T> *__restrict__ tab,
                                               const double *__restrict__ coef, T g, T mlam,
                                               T *smem, T *__restrict__ outG, Acc<T> *acc) {
  using S = EoShape<NQ, BT>;
  constexpr int H = S::H, NQ2 = S::NQ2, NP = S::NP, HP = NP / 2;
  T *s_Ee = smem + S::EPB * 4 * NP, *s_Eo = s_Ee + H * H, *s_w = s_Eo + H * H;
  __syncthreads();
  for (int t = threadIdx.x; t < H * H; t += blockDim.x) {
    s_Ee[t] = tab->Ee[t];
    s_Eo[t] = tab->Eo[t];
  }
  for (int t = threadIdx.x; t < NQ; t += blockDim.x) s_w[t] = tab->w[t];
  const int le = threadIdx.x / NQ2;
  const int ij = threadIdx.x - le * NQ2;
  const int i = ij % NQ, j = ij / NQ;
  const int64_t slot = slot0 + le;
  bool active = le < S::EPB && slot < E;
  const int64_t e = active && order ? (int64_t)order[slot] : slot;
  if (active && !chk(bs_pred_index(e, tab->ne), BS_CHK_OP_ENTRY)) active = false;
  T *U = smem + (le < S::EPB ? le : 0) * 4 * NP;  // u, then the r outputs
  T *Er = U + NP, *Es = U + 2 * NP, *AS = U + 3 * NP;
  T ureg[NQ];
  int32_t gid[FUSED ? NQ : 1];
  if (active) {
    const int64_t base = e * NP + ij;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      T v;
      if (FUSED) {
        int32_t id = __ldcs(ids + base + k * NQ2);
        if (!chk(bs_pred_fused_entry(id, tab->ng), BS_CHK_OP_ENTRY)) id = -1;
        gid[k] = id;
        v = id != -1 ? in[id >= 0 ? id : -2 - id] : T(0);
      } else if (GATHER_IN) {
        int32_t id = __ldcs(ids + base + k * NQ2);
        if (!chk(bs_pred_map_entry(id, tab->ng), BS_CHK_OP_ENTRY)) id = -1;
        v = id >= 0 ? in[id] : T(0);
      } else {
        v = __ldcs(in + base + k * NQ2);
      }
      ureg[k] = v;
      U[ij + k * NQ2] = v;
    }
  }
  __syncthreads();
  // e/o values: threads i < h for the pair (i, N - i) of row j along r; the
  // others for the pair (i - h, N - i + h) of column j along s
  const bool rtask = i < H;
  const int a = rtask ? i : i - H;
  if (active) {
    T *dst = rtask ? Er : Es;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const T u0 = rtask ? U[a + NQ * j + NQ2 * k] : U[j + NQ * a + NQ2 * k];
      const T u1 = rtask ? U[(NQ - 1 - a) + NQ * j + NQ2 * k] : U[j + NQ * (NQ - 1 - a) + NQ2 * k];
      dst[a + H * (j + NQ * k)] = u0 + u1;
      dst[HP + a + H * (j + NQ * k)] = u0 - u1;
    }
  }
  __syncthreads();
  // one output pair per thread and layer: along r into U (u is dead), along s into AS
  if (active) {
    const T *src = rtask ? Er : Es;
    T ee[H], eo[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
      ee[m] = s_Ee[a * H + m];
      eo[m] = s_Eo[a * H + m];
    }
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      T se = T(0), so = T(0);
#pragma unroll
      for (int m = 0; m < H; ++m) {
        se = fmaT(ee[m], src[m + H * (j + NQ * k)], se);
        so = fmaT(eo[m], src[HP + m + H * (j + NQ * k)], so);
      }
      if (rtask) {
        U[a + NQ * j + NQ2 * k] = se + so;
        U[(NQ - 1 - a) + NQ * j + NQ2 * k] = se - so;
      } else {
        AS[j + NQ * a + NQ2 * k] = se + so;
        AS[j + NQ * (NQ - 1 - a) + NQ2 * k] = se - so;
      }
    }
  }
  // along t, from the thread's own column
  T at[NQ];
  if (active) {
    T ev[H], ov[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
      ev[m] = ureg[m] + ureg[NQ - 1 - m];
      ov[m] = ureg[m] - ureg[NQ - 1 - m];
    }
#pragma unroll
    for (int k = 0; k < H; ++k) {
      T se = T(0), so = T(0);
#pragma unroll
      for (int m = 0; m < H; ++m) {
        se = fmaT(s_Ee[k * H + m], ev[m], se);
        so = fmaT(s_Eo[k * H + m], ov[m], so);
      }
      at[k] = se + so;
      at[NQ - 1 - k] = se - so;
    }
  }
  __syncthreads();
  if (!active) return;
  const T cg = (coef ? T(coef[e]) : T(1)) * g;
  const T wij = s_w[i] * s_w[j];
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const T sum = (U[ij + NQ2 * k] + AS[ij + NQ2 * k]) + at[k];
    const T res = (wij * s_w[k]) * fmaT(cg, sum, mlam * ureg[k]);
    if (FUSED) {
      const int32_t id = gid[FUSED ? k : 0];
      if (id >= 0) {
        __stcs(out + e * NP + ij + k * NQ2, res);
      } else if (id != -1) {
        const T v = plus_zero(res);
        __stcs(outG + (-2 - id), v);
        acc->add(ureg[k], v);
      }
    } else {
      __stcs(out + e * NP + ij + k * NQ2, res);
    }
  }
}

template <typename T, int NQ, bool GATHER_IN, bool FUSED>
__global__ void __launch_bounds__(EoShape<NQ>::THREADS)
    k_ax_local_eo(int64_t E, const int32_t *__restrict__ order,
                  const int32_t *__restrict__ ids, const T *__restrict__ in,
                  T *__restrict__ out, const OpTab<T> *__restrict__ tab,
                  const double *__restrict__ coef, T g, T mlam, const CgState *st,
                  T *__restrict__ outG, double *__restrict__ partials) {
  using S = EoShape<NQ>;
  __shared__ T smem[S::SMEM];
  if (cg_halted(st)) return;
  Acc<T> acc;
  ax_elements_eo<T, NQ, GATHER_IN, FUSED>((int64_t)blockIdx.x * S::EPB, E, order, ids, in, out,
                                          tab, coef, g, mlam, smem, outG, &acc);
  if (FUSED && partials) {
    const double part = block_sum<S::THREADS>(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = part;
  }
}

// 1: the element kernels of A p (FP64, FP32, float-float) use the even-odd
// form where it exists (the default); 0: the direct sum factorisation.
extern int g_op_evenodd;

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
#define BS_AXB(NQ)                                                      \
  case NQ:                                                              \
    return use_eo<NQ>() && g_op_evenodd                                 \
               ? (E + EoShape<NQ>::EPB - 1) / EoShape<NQ>::EPB          \
               : (E + OpShape<NQ>::EPB - 1) / OpShape<NQ>::EPB;
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
    if constexpr (use_eo<NQ>()) {                                                        \
      if (g_op_evenodd) {                                                                \
        using Se = EoShape<NQ>;                                                          \
        const int64_t grid = (E + Se::EPB - 1) / Se::EPB;                                \
        k_ax_local_eo<T, NQ, GATHER_IN, FUSED><<<(unsigned)grid, Se::THREADS, 0, s>>>(   \
            E, order, ids, in, out, tab, coef, g, mlam, st, outG, partials);             \
        break;                                                                           \
      }                                                                                  \
    }                                                                                    \
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
  double *d_geo;                  // [7 NL] geometric factors of general hexahedra, or NULL
  bs::OpTab<double> *d_tab;       // FP64 tables
  bs::OpTab<float> *d_tabf;       // FP32 tables
  bs::OpTabFF *d_tabff;           // float-pair tables of the float-float operator
  double *d_ApL;                  // [NL] local operator output (FP64 or FP32 view)
  double *d_vec;                  // 6 x [NG]: r, p, Ap, z, dinv, spare
  bs::CgState *d_state;
  double *d_partials;             // [kMaxPartials]
  double *d_op_partials;          // [E + 1] the fused operator's block partials (<= E blocks)
  unsigned int *d_counter;
  bs::CgState *h_state;           // pinned host mirror for convergence checks
  cudaStream_t cap_stream;        // private stream for graph capture
  cudaGraphExec_t graph;          // cached CG chunk graph
  const void *graph_key[4];       // (x, variant, chunk, map) the graph was made for
  float *d_f32;                   // 4 x [NG + 8] FP32 vectors (refined solver), lazily
  double *d_Lvec;                 // 6 x [NL + 2 rounded up to even] scattered CG vectors, lazily
  uint8_t *d_owner;               // [NL + 16] 1 at the lowest local copy of each node, lazily
  void *d_bj;                     // block-Jacobi tables and per-element flags, lazily
};
