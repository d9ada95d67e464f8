// bs_op_ff.cuh -- the element operator of bs_op.cuh evaluated in float-float
// arithmetic on the FP32 pipes.
//
// GB300 runs FP64 at about 1/64 of its FP32 rate (measured: 627 G DFMA/s
// against 39 T FFMA/s), so the FP64 operator -- 3(N+1) + ~8 FP64 operations
// per local node -- is FP64-pipe bound, far from the HBM roofline.  Here every
// input double u is split exactly, by integer operations (no conversion
// instructions, which share the FP64 pipe), into uh = u truncated to 24
// significant bits and ul = the remaining bits rounded to a float
// (|u - uh - ul| <= 2^-48 |u|); the 1-D stiffness K and the weight products
// w_a w_b are split the same way on the host.  Each contraction
// sum_m K_im u_m is then accumulated as an unevaluated float pair: the product
// of the high parts exactly (FMUL and the FFMA of its rounding error), the
// cross terms Kh ul + Kl uh in a float, and the sum of the high products by
// TwoSum (Knuth).  The error of a node's result is a few units of 2^-46 times
// sum |K| |u| (about 64 times FP64's), far below the tolerances CG is run to.
// The coefficient c_e h/2, the mass term lambda (h/2)^3 w_i w_j w_k u and the
// final sum are float pairs too; per node the FP64 pipe does one addition,
// joining the result's pair.
//
// Inputs with |u| < 2^-102 are taken as zero (so are the low parts below
// float's normal range); |u| >= 2^127 becomes infinite, which CG reports as a
// breakdown.
#pragma once

#include <type_traits>

#include "bs_op.cuh"
#include "bs_op_geo.cuh"

namespace bs {

// (FF, the float pair hi + lo, is defined with the FP32 reductions.)

// Split tables: K = Kh + Kl and W[a*Nq + b] = w_a w_b = Wh + Wl (float
// pairs of the double values), and w_a = wh + wl.
struct OpTabFF {
  float Kh[kMaxNq * kMaxNq], Kl[kMaxNq * kMaxNq];
  float Wh[kMaxNq * kMaxNq], Wl[kMaxNq * kMaxNq];
  float wh[kMaxNq], wl[kMaxNq];
  // the GLL derivative matrix D as float pairs (general hexahedra)
  float Dh[kMaxNq * kMaxNq], Dl[kMaxNq * kMaxNq];
  // the even-odd halves OpTab::Ee, OpTab::Eo as float pairs
  float Eeh[(kMaxNq / 2) * (kMaxNq / 2)], Eel[(kMaxNq / 2) * (kMaxNq / 2)];
  float Eoh[(kMaxNq / 2) * (kMaxNq / 2)], Eol[(kMaxNq / 2) * (kMaxNq / 2)];
  int64_t ne, ng;  // the problem's E and N_G (index checks of the checked build)
};

// x = h + l exactly up to 2^-48 |x| (see the header comment); integer and
// FP32 operations only.
__device__ __forceinline__ FF ff_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned E = (hw >> 20) & 0x7ffu;
  const unsigned sign = hw & 0x80000000u;
  if (E < 921u) return FF{0.f, 0.f};                                  // |x| < 2^-102
  if (E > 1150u) return FF{__uint_as_float(sign | 0x7f800000u), 0.f};  // |x| >= 2^127
  const float h =
      __uint_as_float(sign | ((E - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  // the low 29 bits, rounded to 23, times 2^(E - 1069): base = 2^(E - 1046)
  // as a float; the bit pattern base + rr is base (1 + rr 2^-23), so the
  // difference is rr 2^(E - 1069) exactly (rr = 2^23 carries into the
  // exponent and still gives that value)
  const unsigned rr = ((lw & 0x1fffffffu) + 32u) >> 6;
  const unsigned base = (E - 919u) << 23;
  const float l = __uint_as_float(
      __float_as_uint(__uint_as_float(base + rr) - __uint_as_float(base)) | sign);
  return FF{h, l};
}

// A float as a double by assembling its bits (no conversion instruction):
// normal values exactly, subnormals (below 2^-126) flushed to zero, inf and
// nan kept (exponent 0xff maps to 0x7ff).
__device__ __forceinline__ double ff_widen(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned de = e == 0u ? 0u : (e == 0xffu ? 0x7ffu : e + 896u);
  const unsigned m = e == 0u ? 0u : (u & 0x7fffffu);
  const unsigned hi = (u & 0x80000000u) | (de << 20) | (m >> 3);
  return __hiloint2double((int)hi, (int)(m << 29));
}

// s += (a + al)(b + bl), dropping al bl: the high product exactly (p + e),
// the rest in a float, the high parts summed by TwoSum.
__device__ __forceinline__ void ff_fma(FF &s, float a, float al, float b, float bl) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float c = fmaf(a, bl, fmaf(al, b, e));
  const float t = s.hi + p;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo = s.lo + (err + c);
}

// Dot-product step safe at any scale: acc (a float pair) += a b when both
// lie in [2^-60, 2^60) (products, their rounding errors and the low parts
// then stay normal floats), else dacc = fma(a, b, dacc) on the FP64 pipe;
// zeros and subnormals contribute nothing.  The caller adds dacc to the
// widened pair.
__device__ __forceinline__ void ff_dot_acc(FF &acc, double &dacc, double a, double b) {
  const unsigned ea = ((unsigned)__double2hiint(a) >> 20) & 0x7ffu;
  const unsigned eb = ((unsigned)__double2hiint(b) >> 20) & 0x7ffu;
  if (ea - 963u < 120u && eb - 963u < 120u) {
    const FF x = ff_split(a), y = ff_split(b);
    ff_fma(acc, x.hi, x.lo, y.hi, y.lo);
  } else if (ea != 0u && eb != 0u) {
    dacc = fma(a, b, dacc);
  }
}

// out = A_L in on elements slot0 .. slot0 + EPB - 1, as ax_elements
// (FUSED likewise; the dot product reads p_g again, from cache, in FP64).
template <int NQ, bool GATHER_IN, bool FUSED = false>
__device__ __forceinline__ void ax_elements_ff(int64_t slot0, int64_t E,
                                               const int32_t *__restrict__ order,
                                               const int32_t *__restrict__ ids,
                                               const double *__restrict__ in,
                                               double *__restrict__ out,
                                               const OpTabFF *__restrict__ tab,
                                               const double *__restrict__ coef, double g,
                                               double mlam, float *s_uh_all, float *s_ul_all,
                                               float *s_K, float *s_w,
                                               double *__restrict__ outG = nullptr,
                                               Acc<double> *acc = nullptr) {
  static_assert(!FUSED || GATHER_IN, "the fused operator reads its input through the map");
  using S = OpShape<NQ>;
  constexpr int NQ2 = NQ * NQ;
  float *s_Kh = s_K, *s_Kl = s_K + NQ2, *s_Wh = s_K + 2 * NQ2, *s_Wl = s_K + 3 * NQ2;
  __syncthreads();
  for (int t = threadIdx.x; t < NQ2; t += blockDim.x) {
    const int a = t / NQ, b = t % NQ;
    s_Kh[t] = tab->Kh[a * NQ + b];
    s_Kl[t] = tab->Kl[a * NQ + b];
    s_Wh[t] = tab->Wh[a * NQ + b];
    s_Wl[t] = tab->Wl[a * NQ + b];
  }
  for (int t = threadIdx.x; t < NQ; t += blockDim.x) {
    s_w[t] = tab->wh[t];
    s_w[NQ + t] = tab->wl[t];
  }
  const int le = threadIdx.x / NQ2;
  const int ij = threadIdx.x - le * NQ2;
  const int i = ij % NQ, j = ij / NQ;
  const int64_t slot = slot0 + le;
  bool active = le < S::EPB && slot < E;
  const int64_t e = active && order ? (int64_t)order[slot] : slot;
  if (active && !chk(bs_pred_index(e, tab->ne), BS_CHK_OP_ENTRY)) active = false;
  float *uh = s_uh_all + (le < S::EPB ? le : 0) * S::NP;
  float *ul = s_ul_all + (le < S::EPB ? le : 0) * S::NP;
  float rh[NQ], rl[NQ];
  int32_t gid[FUSED ? NQ : 1];
  if (active) {
    const int64_t base = e * S::NP + ij;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      double v;
      if (FUSED) {
        int32_t id = __ldcs(ids + base + k * NQ2);
        if (!chk(bs_pred_fused_entry(id, tab->ng), BS_CHK_OP_ENTRY)) id = -1;
        gid[k] = id;
        v = id != -1 ? in[id >= 0 ? id : -2 - id] : 0.0;
      } else if (GATHER_IN) {
        int32_t id = __ldcs(ids + base + k * NQ2);
        if (!chk(bs_pred_map_entry(id, tab->ng), BS_CHK_OP_ENTRY)) id = -1;
        v = id >= 0 ? in[id] : 0.0;
      } else {
        v = __ldcs(in + base + k * NQ2);
      }
      const FF f = ff_split(v);
      rh[k] = f.hi;
      rl[k] = f.lo;
      uh[ij + k * NQ2] = f.hi;
      ul[ij + k * NQ2] = f.lo;
    }
  }
  __syncthreads();
  if (!active) return;
  // c_e h/2 and lambda (h/2)^3 w_i w_j as float pairs (two FP64 products and
  // their splits per thread, not per node)
  const FF cg = ff_split((coef ? coef[e] : 1.0) * g);
  const FF ml = ff_split(mlam);
  FF mwij{0.f, 0.f};
  ff_fma(mwij, ml.hi, ml.lo, s_Wh[i * NQ + j], s_Wl[i * NQ + j]);
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    FF ar{0.f, 0.f}, as{0.f, 0.f}, at{0.f, 0.f};
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      const int lr = m + NQ * j + NQ2 * k, ls = i + NQ * m + NQ2 * k;
      ff_fma(ar, s_Kh[i * NQ + m], s_Kl[i * NQ + m], uh[lr], ul[lr]);
      ff_fma(as, s_Kh[j * NQ + m], s_Kl[j * NQ + m], uh[ls], ul[ls]);
      ff_fma(at, s_Kh[k * NQ + m], s_Kl[k * NQ + m], rh[m], rl[m]);
    }
    // (w_j w_k) ar + (w_i w_k) as + (w_i w_j) at
    FF t{0.f, 0.f};
    ff_fma(t, s_Wh[j * NQ + k], s_Wl[j * NQ + k], ar.hi, ar.lo);
    ff_fma(t, s_Wh[i * NQ + k], s_Wl[i * NQ + k], as.hi, as.lo);
    ff_fma(t, s_Wh[i * NQ + j], s_Wl[i * NQ + j], at.hi, at.lo);
    // c_e h/2 stiff + (lambda (h/2)^3 w_i w_j w_k) u_ijk
    FF mk{0.f, 0.f};
    ff_fma(mk, mwij.hi, mwij.lo, s_w[k], s_w[NQ + k]);
    FF o{0.f, 0.f};
    ff_fma(o, cg.hi, cg.lo, t.hi, t.lo);
    ff_fma(o, mk.hi, mk.lo, rh[k], rl[k]);
    const double res = ff_widen(o.hi) + ff_widen(o.lo);
    if (FUSED) {
      const int32_t id = gid[FUSED ? k : 0];
      if (id >= 0) {
        __stcs(out + e * S::NP + ij + k * NQ2, res);
      } else if (id != -1) {
        const double v = plus_zero(res);
        __stcs(outG + (-2 - id), v);
        acc->add(__ldg(in + (-2 - id)), v);
      }
    } else {
      __stcs(out + e * S::NP + ij + k * NQ2, res);
    }
  }
}

// a + b for unevaluated float pairs: TwoSum of the high parts, low parts
// and the rounding error added (not renormalised, as in ff_fma).
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b.hi - bb);
  return FF{s, (a.lo + b.lo) + err};
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }

// The even-odd form of bs_op.cuh (ax_elements_eo) in float-float arithmetic:
// the same phases, every value a float pair (e/o values by ff_add, the
// half-length contractions by ff_fma), result W3 (c (h/2) sum + lambda
// (h/2)^3 u) joined into a double.  smem holds EoShapeFF<NQ, BT>::SMEM floats.
template <int NQ, int BT = 128>
struct EoShapeFF {
  using S = EoShape<NQ, BT>;
  static constexpr int SMEM = S::EPB * 8 * S::NP + 4 * S::H * S::H + 2 * NQ;
};

template <int NQ, bool GATHER_IN, bool FUSED, int BT = 128>
__device__ __forceinline__ void ax_elements_ff_eo(int64_t slot0, int64_t E,
                                                  const int32_t *__restrict__ order,
                                                  const int32_t *__restrict__ ids,
                                                  const double *__restrict__ in,
                                                  double *__restrict__ out,
                                                  const OpTabFF *__restrict__ tab,
                                                  const double *__restrict__ coef, double g,
                                                  double mlam, float *smem,
                                                  double *__restrict__ outG,
                                                  Acc<double> *acc) {
  using S = EoShape<NQ, BT>;
  constexpr int H = S::H, NQ2 = S::NQ2, NP = S::NP, HP = NP / 2, HH = H * H;
  // float pairs kept as float2 (hi, lo): one 8-byte shared access per value
  // (smem is 8-byte aligned)
  float2 *sm2 = reinterpret_cast<float2 *>(smem);
  float2 *s_Ee = sm2 + S::EPB * 4 * NP, *s_Eo = s_Ee + HH, *s_w = s_Eo + HH;
  __syncthreads();
  for (int t = threadIdx.x; t < HH; t += blockDim.x) {
    s_Ee[t] = make_float2(tab->Eeh[t], tab->Eel[t]);
    s_Eo[t] = make_float2(tab->Eoh[t], tab->Eol[t]);
  }
  for (int t = threadIdx.x; t < NQ; t += blockDim.x) s_w[t] = make_float2(tab->wh[t], tab->wl[t]);
  const int le = threadIdx.x / NQ2;
  const int ij = threadIdx.x - le * NQ2;
  const int i = ij % NQ, j = ij / NQ;
  const int64_t slot = slot0 + le;
  bool active = le < S::EPB && slot < E;
  const int64_t e = active && order ? (int64_t)order[slot] : slot;
  if (active && !chk(bs_pred_index(e, tab->ne), BS_CHK_OP_ENTRY)) active = false;
  float2 *U = sm2 + (le < S::EPB ? le : 0) * 4 * NP;  // u, then the r outputs
  float2 *Er = U + NP, *Es = U + 2 * NP, *AS = U + 3 * NP;
  float rh[NQ], rl[NQ];
  int32_t gid[FUSED ? NQ : 1];
  if (active) {
    const int64_t base = e * NP + ij;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      double v;
      if (FUSED) {
        int32_t id = __ldcs(ids + base + k * NQ2);
        if (!chk(bs_pred_fused_entry(id, tab->ng), BS_CHK_OP_ENTRY)) id = -1;
        gid[k] = id;
        v = id != -1 ? in[id >= 0 ? id : -2 - id] : 0.0;
      } else if (GATHER_IN) {
        int32_t id = __ldcs(ids + base + k * NQ2);
        if (!chk(bs_pred_map_entry(id, tab->ng), BS_CHK_OP_ENTRY)) id = -1;
        v = id >= 0 ? in[id] : 0.0;
      } else {
        v = __ldcs(in + base + k * NQ2);
      }
      const FF f = ff_split(v);
      rh[k] = f.hi;
      rl[k] = f.lo;
      U[ij + k * NQ2] = make_float2(f.hi, f.lo);
    }
  }
  __syncthreads();
  const bool rtask = i < H;
  const int a = rtask ? i : i - H;
  if (active) {
    float2 *dst = rtask ? Er : Es;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const int l0 = rtask ? a + NQ * j + NQ2 * k : j + NQ * a + NQ2 * k;
      const int l1 = rtask ? (NQ - 1 - a) + NQ * j + NQ2 * k : j + NQ * (NQ - 1 - a) + NQ2 * k;
      const float2 x0 = U[l0], x1 = U[l1];
      const FF u0{x0.x, x0.y}, u1{x1.x, x1.y};
      const FF ev = ff_add(u0, u1), ov = ff_add(u0, ff_neg(u1));
      const int d = a + H * (j + NQ * k);
      dst[d] = make_float2(ev.hi, ev.lo);
      dst[HP + d] = make_float2(ov.hi, ov.lo);
    }
  }
  __syncthreads();
  if (active) {
    const float2 *src = rtask ? Er : Es;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      FF se{0.f, 0.f}, so{0.f, 0.f};
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const int d = m + H * (j + NQ * k);
        const float2 ce = s_Ee[a * H + m], co = s_Eo[a * H + m], xe = src[d], xo = src[HP + d];
        ff_fma(se, ce.x, ce.y, xe.x, xe.y);
        ff_fma(so, co.x, co.y, xo.x, xo.y);
      }
      const FF p = ff_add(se, so), q = ff_add(se, ff_neg(so));
      if (rtask) {
        const int l0 = a + NQ * j + NQ2 * k, l1 = (NQ - 1 - a) + NQ * j + NQ2 * k;
        U[l0] = make_float2(p.hi, p.lo);
        U[l1] = make_float2(q.hi, q.lo);
      } else {
        const int l0 = j + NQ * a + NQ2 * k, l1 = j + NQ * (NQ - 1 - a) + NQ2 * k;
        AS[l0] = make_float2(p.hi, p.lo);
        AS[l1] = make_float2(q.hi, q.lo);
      }
    }
  }
  FF at[NQ];
  if (active) {
    FF ev[H], ov[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
      const FF u0{rh[m], rl[m]}, u1{rh[NQ - 1 - m], rl[NQ - 1 - m]};
      ev[m] = ff_add(u0, u1);
      ov[m] = ff_add(u0, ff_neg(u1));
    }
#pragma unroll
    for (int k = 0; k < H; ++k) {
      FF se{0.f, 0.f}, so{0.f, 0.f};
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const float2 ce = s_Ee[k * H + m], co = s_Eo[k * H + m];
        ff_fma(se, ce.x, ce.y, ev[m].hi, ev[m].lo);
        ff_fma(so, co.x, co.y, ov[m].hi, ov[m].lo);
      }
      at[k] = ff_add(se, so);
      at[NQ - 1 - k] = ff_add(se, ff_neg(so));
    }
  }
  __syncthreads();
  if (!active) return;
  const FF cg = ff_split((coef ? coef[e] : 1.0) * g);
  const FF ml = ff_split(mlam);
  FF wij{0.f, 0.f};
  ff_fma(wij, s_w[i].x, s_w[i].y, s_w[j].x, s_w[j].y);
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const int l = ij + NQ2 * k;
    const float2 uu = U[l], aa = AS[l];
    const FF sum = ff_add(ff_add(FF{uu.x, uu.y}, FF{aa.x, aa.y}), at[k]);
    FF o{0.f, 0.f};
    ff_fma(o, cg.hi, cg.lo, sum.hi, sum.lo);
    ff_fma(o, ml.hi, ml.lo, rh[k], rl[k]);
    FF w3{0.f, 0.f};
    ff_fma(w3, wij.hi, wij.lo, s_w[k].x, s_w[k].y);
    FF r{0.f, 0.f};
    ff_fma(r, w3.hi, w3.lo, o.hi, o.lo);
    const double res = ff_widen(r.hi) + ff_widen(r.lo);
    if (FUSED) {
      const int32_t id = gid[FUSED ? k : 0];
      if (id >= 0) {
        __stcs(out + e * NP + l, res);
      } else if (id != -1) {
        const double v = plus_zero(res);
        __stcs(outG + (-2 - id), v);
        acc->add(__ldg(in + (-2 - id)), v);
      }
    } else {
      __stcs(out + e * NP + l, res);
    }
  }
}

template <int NQ, bool GATHER_IN, bool FUSED>
__global__ void __launch_bounds__(EoShape<NQ>::THREADS)
    k_ax_local_ff_eo(int64_t E, const int32_t *__restrict__ order,
                     const int32_t *__restrict__ ids, const double *__restrict__ in,
                     double *__restrict__ out, const OpTabFF *__restrict__ tab,
                     const double *__restrict__ coef, double g, double mlam,
                     const CgState *st, double *__restrict__ outG,
                     double *__restrict__ partials) {
  using S = EoShape<NQ>;
  __shared__ __align__(16) float smem[EoShapeFF<NQ>::SMEM];
  if (cg_halted(st)) return;
  Acc<double> acc;
  ax_elements_ff_eo<NQ, GATHER_IN, FUSED>((int64_t)blockIdx.x * S::EPB, E, order, ids, in, out,
                                          tab, coef, g, mlam, smem, outG, &acc);
  if (FUSED && partials) {
    const double part = block_sum<S::THREADS>(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = part;
  }
}

template <int NQ, bool GATHER_IN, bool FUSED>
__global__ void __launch_bounds__(OpShape<NQ>::THREADS)
    k_ax_local_ff(int64_t E, const int32_t *__restrict__ order, const int32_t *__restrict__ ids,
                  const double *__restrict__ in, double *__restrict__ out,
                  const OpTabFF *__restrict__ tab, const double *__restrict__ coef, double g,
                  double mlam, const CgState *st, double *__restrict__ outG,
                  double *__restrict__ partials) {
  using S = OpShape<NQ>;
  __shared__ float s_uh[S::EPB * S::NP];
  __shared__ float s_ul[S::EPB * S::NP];
  __shared__ float s_K[4 * NQ * NQ];
  __shared__ float s_w[2 * NQ];
  if (cg_halted(st)) return;
  Acc<double> acc;
  ax_elements_ff<NQ, GATHER_IN, FUSED>((int64_t)blockIdx.x * S::EPB, E, order, ids, in, out,
                                       tab, coef, g, mlam, s_uh, s_ul, s_K, s_w, outG, &acc);
  if (FUSED && partials) {
    const double part = block_sum<S::THREADS>(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = part;
  }
}

template <bool GATHER_IN, bool FUSED = false>
int launch_ax_local_ff(int N, int64_t E, const int32_t *order, const int32_t *ids,
                       const double *in, double *out, const OpTabFF *tab, const double *coef,
                       double g, double mlam, const CgState *st, cudaStream_t s,
                       double *outG = nullptr, double *partials = nullptr) {
  if (E == 0) return BS_OK;
#define BS_AXFF_CASE(NQ)                                                              \
  case NQ: {                                                                          \
    if constexpr (use_eo<NQ>()) {                                                     \
      if (g_op_evenodd) {                                                             \
        using Se = EoShape<NQ>;                                                       \
        const int64_t grid = (E + Se::EPB - 1) / Se::EPB;                             \
        k_ax_local_ff_eo<NQ, GATHER_IN, FUSED><<<(unsigned)grid, Se::THREADS, 0, s>>>( \
            E, order, ids, in, out, tab, coef, g, mlam, st, outG, partials);          \
        break;                                                                        \
      }                                                                               \
    }                                                                                 \
    using Sh = OpShape<NQ>;                                                           \
    const int64_t grid = (E + Sh::EPB - 1) / Sh::EPB;                                 \
    k_ax_local_ff<NQ, GATHER_IN, FUSED><<<(unsigned)grid, Sh::THREADS, 0, s>>>(       \
        E, order, ids, in, out, tab, coef, g, mlam, st, outG, partials);              \
    break;                                                                            \
  }
  switch (N + 1) {
    BS_AXFF_CASE(2)
    BS_AXFF_CASE(3)
    BS_AXFF_CASE(4)
    BS_AXFF_CASE(5)
    BS_AXFF_CASE(6)
    BS_AXFF_CASE(7)
    BS_AXFF_CASE(8)
    BS_AXFF_CASE(9)
    BS_AXFF_CASE(10)
    BS_AXFF_CASE(11)
    BS_AXFF_CASE(12)
    BS_AXFF_CASE(13)
    BS_AXFF_CASE(14)
    BS_AXFF_CASE(15)
    BS_AXFF_CASE(16)
    default:
      return fail(BS_ERR_ARG, "degree %d unsupported", N);
  }
#undef BS_AXFF_CASE
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// ---------------------------------------------------------------- general hexahedra

// The general-hexahedron operator of bs_op_geo.cuh in float-float
// arithmetic: u, D and the six factors of every node split into float pairs
// (the factors on the fly, by integer operations), the gradient, the flux
// G grad u and the transposed derivative accumulated by ff_fma, the mass term
// from one FP64 product lambda M per node; the result joined into a double.
// Same thread mapping and phases as k_ax_geo.
template <int NQ, bool GATHER_IN>
__global__ void __launch_bounds__(GeoShape<NQ>::THREADS)
    k_ax_geo_ff(int64_t E, int64_t NL, const int32_t *__restrict__ order,
                const int32_t *__restrict__ ids, const double *__restrict__ in,
                double *__restrict__ out, const OpTabFF *__restrict__ tab,
                const double *__restrict__ coef, const double *__restrict__ geo, double lambda,
                const CgState *st) {
  using S = GeoShape<NQ>;
  constexpr int NQ2 = S::NQ2, NP = S::NP;
  __shared__ float s_uh[S::EPB * NP], s_ul[S::EPB * NP];
  __shared__ float s_frh[S::EPB * NP], s_frl[S::EPB * NP];
  __shared__ float s_fsh[S::EPB * NP], s_fsl[S::EPB * NP];
  __shared__ float s_Dh[NQ2], s_Dl[NQ2];
  if (cg_halted(st)) return;
  for (int t = threadIdx.x; t < NQ2; t += blockDim.x) {
    s_Dh[t] = tab->Dh[t];
    s_Dl[t] = tab->Dl[t];
  }
  const int le = threadIdx.x / NQ2;
  const int ij = threadIdx.x - le * NQ2;
  const int i = ij % NQ, j = ij / NQ;
  const int64_t slot = (int64_t)blockIdx.x * S::EPB + le;
  bool active = le < S::EPB && slot < E;
  const int64_t e = active && order ? (int64_t)order[slot] : slot;
  if (active && !chk(bs_pred_index(e, tab->ne), BS_CHK_OP_ENTRY)) active = false;
  const int off = (le < S::EPB ? le : 0) * NP;
  float *uh = s_uh + off, *ul = s_ul + off;
  float *frh = s_frh + off, *frl = s_frl + off, *fsh = s_fsh + off, *fsl = s_fsl + off;
  float rh[NQ], rl[NQ];
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
      const FF f = ff_split(v);
      rh[k] = f.hi;
      rl[k] = f.lo;
      uh[ij + k * NQ2] = f.hi;
      ul[ij + k * NQ2] = f.lo;
    }
  }
  __syncthreads();
  FF ft[NQ];
  if (active) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      FF ur{0.f, 0.f}, us{0.f, 0.f}, ut{0.f, 0.f};
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        const int lr = m + NQ * j + NQ2 * k, ls = i + NQ * m + NQ2 * k;
        ff_fma(ur, s_Dh[i * NQ + m], s_Dl[i * NQ + m], uh[lr], ul[lr]);
        ff_fma(us, s_Dh[j * NQ + m], s_Dl[j * NQ + m], uh[ls], ul[ls]);
        ff_fma(ut, s_Dh[k * NQ + m], s_Dl[k * NQ + m], rh[m], rl[m]);
      }
      const int64_t l = e * NP + ij + k * NQ2;
      const FF g0 = ff_split(__ldcs(geo + l)), g1 = ff_split(__ldcs(geo + NL + l));
      const FF g2 = ff_split(__ldcs(geo + 2 * NL + l)), g3 = ff_split(__ldcs(geo + 3 * NL + l));
      const FF g4 = ff_split(__ldcs(geo + 4 * NL + l)), g5 = ff_split(__ldcs(geo + 5 * NL + l));
      FF fr{0.f, 0.f}, fs{0.f, 0.f}, fq{0.f, 0.f};
      ff_fma(fr, g0.hi, g0.lo, ur.hi, ur.lo);
      ff_fma(fr, g1.hi, g1.lo, us.hi, us.lo);
      ff_fma(fr, g2.hi, g2.lo, ut.hi, ut.lo);
      ff_fma(fs, g1.hi, g1.lo, ur.hi, ur.lo);
      ff_fma(fs, g3.hi, g3.lo, us.hi, us.lo);
      ff_fma(fs, g4.hi, g4.lo, ut.hi, ut.lo);
      ff_fma(fq, g2.hi, g2.lo, ur.hi, ur.lo);
      ff_fma(fq, g4.hi, g4.lo, us.hi, us.lo);
      ff_fma(fq, g5.hi, g5.lo, ut.hi, ut.lo);
      frh[ij + k * NQ2] = fr.hi;
      frl[ij + k * NQ2] = fr.lo;
      fsh[ij + k * NQ2] = fs.hi;
      fsl[ij + k * NQ2] = fs.lo;
      ft[k] = fq;
    }
  }
  __syncthreads();
  if (!active) return;
  const FF cg = ff_split(coef ? coef[e] : 1.0);
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    FF acc{0.f, 0.f};
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      const int lr = m + NQ * j + NQ2 * k, ls = i + NQ * m + NQ2 * k;
      ff_fma(acc, s_Dh[m * NQ + i], s_Dl[m * NQ + i], frh[lr], frl[lr]);
      ff_fma(acc, s_Dh[m * NQ + j], s_Dl[m * NQ + j], fsh[ls], fsl[ls]);
      ff_fma(acc, s_Dh[m * NQ + k], s_Dl[m * NQ + k], ft[m].hi, ft[m].lo);
    }
    const int64_t l = e * NP + ij + k * NQ2;
    const FF lm = ff_split(lambda * __ldcs(geo + 6 * NL + l));
    FF o{0.f, 0.f};
    ff_fma(o, cg.hi, cg.lo, acc.hi, acc.lo);
    ff_fma(o, lm.hi, lm.lo, rh[k], rl[k]);
    __stcs(out + l, ff_widen(o.hi) + ff_widen(o.lo));
  }
}

template <bool GATHER_IN>
int launch_ax_geo_ff(int N, int64_t E, int64_t NL, const int32_t *order, const int32_t *ids,
                     const double *in, double *out, const OpTabFF *tab, const double *coef,
                     const double *geo, double lambda, const CgState *st, cudaStream_t s) {
  if (E == 0) return BS_OK;
#define BS_AXGF_CASE(NQ)                                                                 \
  case NQ: {                                                                             \
    using Sh = GeoShape<NQ>;                                                             \
    const int64_t grid = (E + Sh::EPB - 1) / Sh::EPB;                                    \
    k_ax_geo_ff<NQ, GATHER_IN><<<(unsigned)grid, Sh::THREADS, 0, s>>>(                   \
        E, NL, order, ids, in, out, tab, coef, geo, lambda, st);                         \
    break;                                                                               \
  }
  switch (N + 1) {
    BS_AXGF_CASE(2)
    BS_AXGF_CASE(3)
    BS_AXGF_CASE(4)
    BS_AXGF_CASE(5)
    BS_AXGF_CASE(6)
    BS_AXGF_CASE(7)
    BS_AXGF_CASE(8)
    BS_AXGF_CASE(9)
    BS_AXGF_CASE(10)
    BS_AXGF_CASE(11)
    BS_AXGF_CASE(12)
    default:
      return fail(BS_ERR_ARG, "degree %d unsupported with geometric factors", N);
  }
#undef BS_AXGF_CASE
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// 1: A p through the fused element kernel and the gather of the shared rows;
// 0 (the default): element kernel, then the gather of every row.
extern int g_op_fusion;

// Ap = A p for a global p (FP64 or FP32 tables; ff: the float-float element
// kernel, FP64 only).  DOT: ep(p . Ap), reduced in the gather's pass (and,
// fused, in the element kernel's epilogue for the single-copy nodes).
template <typename T, bool DOT, class Ep>
int apply_A_global(const bs_problem *P, bool ff, const OpTab<T> *tab, const T *p, T *Ap, T *ApL,
                   T g, T mlam, Ep ep, const CgState *st, cudaStream_t s) {
  const bs_map *m = P->map;
  if (P->d_geo) {  // general hexahedra: FP64 or float-float, unfused
    if constexpr (std::is_same<T, double>::value) {
      if (int rc = ff ? launch_ax_geo_ff<true>(P->N, m->E, m->NL, m->d_elem_order, m->d_ids, p,
                                               ApL, P->d_tabff, P->d_coef, P->d_geo, P->lambda,
                                               st, s)
                      : launch_ax_geo<true>(P->N, m->E, m->NL, m->d_elem_order, m->d_ids, p, ApL,
                                            P->d_tab, P->d_coef, P->d_geo, P->lambda, st, s))
        return rc;
      return launch_gather<T, DOT, Ep>(m, ApL, Ap, DOT ? p : nullptr, P->d_partials,
                                       P->d_counter, ep, st, s);
    } else {
      return fail(BS_ERR_ARG, "FP32 operator not available with geometric factors");
    }
  }
  const bool fused = g_op_fusion != 0;
  const int32_t *ids = fused ? m->d_ids_f : m->d_ids;
  double *opp = fused && DOT ? P->d_op_partials : nullptr;
  int rc;
  if constexpr (std::is_same<T, double>::value) {
    if (ff)
      rc = fused ? launch_ax_local_ff<true, true>(P->N, m->E, m->d_elem_order, ids, p, ApL,
                                                  P->d_tabff, P->d_coef, g, mlam, st, s, Ap, opp)
                 : launch_ax_local_ff<true>(P->N, m->E, m->d_elem_order, ids, p, ApL, P->d_tabff,
                                            P->d_coef, g, mlam, st, s);
    else
      rc = fused ? launch_ax_local<T, true, true>(P->N, m->E, m->d_elem_order, ids, p, ApL, tab,
                                                  P->d_coef, g, mlam, st, s, Ap, opp)
                 : launch_ax_local<T, true>(P->N, m->E, m->d_elem_order, ids, p, ApL, tab,
                                            P->d_coef, g, mlam, st, s);
  } else {
    if (ff) return fail(BS_ERR_ARG, "the float-float operator is FP64 only");
    rc = fused ? launch_ax_local<T, true, true>(P->N, m->E, m->d_elem_order, ids, p, ApL, tab,
                                                P->d_coef, g, mlam, st, s, Ap, opp)
               : launch_ax_local<T, true>(P->N, m->E, m->d_elem_order, ids, p, ApL, tab,
                                          P->d_coef, g, mlam, st, s);
  }
  if (rc) return rc;
  if (!fused)
    return launch_gather<T, DOT, Ep>(m, ApL, Ap, DOT ? p : nullptr, P->d_partials, P->d_counter,
                                     ep, st, s);
  return launch_gather_rows<T, DOT, Ep>(m, fused, ApL, Ap, DOT ? p : nullptr, P->d_partials,
                                        P->d_counter, opp, opp ? ax_blocks(P->N, m->E) : 0, ep,
                                        st, s);
}

}  // namespace bs
