// bs_op_geo.cuh -- the operator A = Z^T (c S_L + lambda M_L) Z on general
// (trilinear) hexahedra: the non-affine geometric factors that the paper's
// gather/scatter discussion allows for (Sec. 5) but its affine BP setting
// does not need.
//
// With J = dx/dr at a GLL node q of element e and w_q the product of the
// three GLL weights, the weak form gives
//   (A_e u)_n = c_e sum_q grad_r l_n(q)^T G_q grad_r u(q) + lambda M_n u_n,
//   G_q = w_q det J J^-1 J^-T (symmetric, six entries),  M_n = w_n det J(n).
// G and M are computed once per problem on the host from the element corners
// and kept in HBM, structure of arrays: d_geo[f * N_L + l], f = 0..5 for
// G_rr, G_rs, G_rt, G_ss, G_st, G_tt and f = 6 for M.  The kernel maps one
// thread to a column (i, j) of an element and walks k: the reference gradient
// (3 (N+1) multiply-adds per node), the flux G grad u (9), then the
// transposed derivative (3 (N+1)) after a block barrier, with the r and s
// fluxes in shared memory and the t flux in registers.  About 6 (N+1) + 12
// FP64 operations and 56 bytes of factors per local node: FP64-pipe bound on
// GB300 (the factors alone would take 0.5 ms of HBM time at N = 7 on 48^3).
// Degrees 1..11.  A float-float form of the same kernel is in bs_op_ff.cuh.
#pragma once

#include "bs_op.cuh"

namespace bs {

constexpr int kGeoMaxNq = 12;
constexpr int kGeoFactors = 7;

template <int NQ>
struct GeoShape {
  static constexpr int NQ2 = NQ * NQ;
  static constexpr int NP = NQ * NQ2;
  static constexpr int EPB = NQ2 >= 128 ? 1 : 128 / NQ2;
  static constexpr int THREADS = ((EPB * NQ2 + 31) / 32) * 32;
};

template <int NQ, bool GATHER_IN>
__global__ void __launch_bounds__(GeoShape<NQ>::THREADS)
    k_ax_geo(int64_t E, int64_t NL, const int32_t *__restrict__ order,
             const int32_t *__restrict__ ids, const double *__restrict__ in,
             double *__restrict__ out, const OpTab<double> *__restrict__ tab,
             const double *__restrict__ coef, const double *__restrict__ geo, double lambda,
             const CgState *st) {
  using S = GeoShape<NQ>;
  constexpr int NQ2 = S::NQ2, NP = S::NP;
  __shared__ double s_u[S::EPB * NP], s_fr[S::EPB * NP], s_fs[S::EPB * NP];
  __shared__ double s_D[NQ2];
  if (cg_halted(st)) return;
  for (int t = threadIdx.x; t < NQ2; t += blockDim.x) s_D[t] = tab->D[t];
  const int le = threadIdx.x / NQ2;
  const int ij = threadIdx.x - le * NQ2;
  const int i = ij % NQ, j = ij / NQ;
  const int64_t slot = (int64_t)blockIdx.x * S::EPB + le;
  bool active = le < S::EPB && slot < E;
  const int64_t e = active && order ? (int64_t)order[slot] : slot;
  if (active && !chk(bs_pred_index(e, tab->ne), BS_CHK_OP_ENTRY)) active = false;
  const int off = (le < S::EPB ? le : 0) * NP;
  double *u = s_u + off, *fr = s_fr + off, *fs = s_fs + off;
  double ureg[NQ], ft[NQ];
  if (active) {
    const int64_t base = e * NP + ij;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      double v;
      if (GATHER_IN) {
        int32_t id = __ldcs(ids + base + k * NQ2);
        if (!chk(bs_pred_map_entry(id, tab->ng), BS_CHK_OP_ENTRY)) id = -1;
        v = id >= 0 ? in[id] : 0.0;
      } else {
        v = __ldcs(in + base + k * NQ2);
      }
      ureg[k] = v;
      u[ij + k * NQ2] = v;
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      double ur = 0.0, us = 0.0, ut = 0.0;
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        ur = fma(s_D[i * NQ + m], u[m + NQ * j + NQ2 * k], ur);
        us = fma(s_D[j * NQ + m], u[i + NQ * m + NQ2 * k], us);
        ut = fma(s_D[k * NQ + m], ureg[m], ut);
      }
      const int64_t l = e * NP + ij + k * NQ2;
      const double g0 = __ldcs(geo + l), g1 = __ldcs(geo + NL + l), g2 = __ldcs(geo + 2 * NL + l);
      const double g3 = __ldcs(geo + 3 * NL + l), g4 = __ldcs(geo + 4 * NL + l);
      const double g5 = __ldcs(geo + 5 * NL + l);
      fr[ij + k * NQ2] = fma(g0, ur, fma(g1, us, g2 * ut));
      fs[ij + k * NQ2] = fma(g1, ur, fma(g3, us, g4 * ut));
      ft[k] = fma(g2, ur, fma(g4, us, g5 * ut));
    }
  }
  __syncthreads();
  if (!active) return;
  const double ce = coef ? coef[e] : 1.0;
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      s = fma(s_D[m * NQ + i], fr[m + NQ * j + NQ2 * k], s);
      s = fma(s_D[m * NQ + j], fs[i + NQ * m + NQ2 * k], s);
      s = fma(s_D[m * NQ + k], ft[m], s);
    }
    const int64_t l = e * NP + ij + k * NQ2;
    __stcs(out + l, fma(ce, s, lambda * (__ldcs(geo + 6 * NL + l) * ureg[k])));
  }
}

template <bool GATHER_IN>
int launch_ax_geo(int N, int64_t E, int64_t NL, const int32_t *order, const int32_t *ids,
                  const double *in, double *out, const OpTab<double> *tab, const double *coef,
                  const double *geo, double lambda, const CgState *st, cudaStream_t s) {
  if (E == 0) return BS_OK;
#define BS_AXG_CASE(NQ)                                                                  \
  case NQ: {                                                                             \
    using Sh = GeoShape<NQ>;                                                             \
    const int64_t grid = (E + Sh::EPB - 1) / Sh::EPB;                                    \
    k_ax_geo<NQ, GATHER_IN><<<(unsigned)grid, Sh::THREADS, 0, s>>>(                      \
        E, NL, order, ids, in, out, tab, coef, geo, lambda, st);                         \
    break;                                                                               \
  }
  switch (N + 1) {
    BS_AXG_CASE(2)
    BS_AXG_CASE(3)
    BS_AXG_CASE(4)
    BS_AXG_CASE(5)
    BS_AXG_CASE(6)
    BS_AXG_CASE(7)
    BS_AXG_CASE(8)
    BS_AXG_CASE(9)
    BS_AXG_CASE(10)
    BS_AXG_CASE(11)
    BS_AXG_CASE(12)
    default:
      return fail(BS_ERR_ARG, "degree %d unsupported with geometric factors", N);
  }
#undef BS_AXG_CASE
  BS_LAUNCH_CHECK();
  return BS_OK;
}

}  // namespace bs
