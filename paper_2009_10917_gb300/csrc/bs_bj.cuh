// bs_bj.cuh -- the element-interior block-Jacobi preconditioner of
// BS_CG_BLOCK_JACOBI: z = D^-1 r, except that on every element whose interior
// nodes belong to it alone the interior block of the element matrix is
// inverted exactly, z_I = A_II^-1 r_I.  This is the map the learned
// preconditioner is trained to imitate (its targets are A_II^-1 r_I), in
// closed form.
//
// On an affine cube A_II = c_e (h/2) (K x W x W + W x K x W + W x W x K)_II
// + lambda (h/2)^3 (W x W x W)_II is a sum of Kronecker products of the 1-D
// interior blocks K_ii and W_ii, so the generalized eigenvectors of
// K_ii v = mu W_ii v (V^T W_ii V = I) diagonalise it (the fast diagonalisation
// method of Lynch, Rice & Thomas, 1964):
//   A_II^-1 = (V x V x V) diag(1 / (c_e (h/2)(mu_a + mu_b + mu_c) + lambda (h/2)^3))
//             (V x V x V)^T,
// i.e. three 1-D transforms, a diagonal scaling and three transforms back,
// 6 (N-1) multiply-adds per interior node.  They run in float-float
// arithmetic on the FP32 pipes (64 times GB300's FP64 rate): inputs split
// exactly into float pairs by integer operations, error-free products and
// TwoSum accumulation, about 2^-46 relative.  Plain FP32 would not do: CG with
// a preconditioner perturbed at 1e-7 lost up to a third more iterations at
// tolerance 1e-10 on low degrees.  Residuals whose RMS lies outside
// [2^-120, 2^120] are scaled by a power of two first (exact both ways).
#pragma once

#include <cmath>
#include <vector>

#include "bs_op_ff.cuh"

namespace bs {

constexpr int kBjMaxNi = 8;  // interior points per direction: N <= 9

// V[m * ni + a] = component m of eigenvector a and M[a + ni (b + ni c)] =
// mu_a + mu_b + mu_c, as float pairs (h + l) of the double values.
struct BjTab {
  float Vh[kBjMaxNi * kBjMaxNi], Vl[kBjMaxNi * kBjMaxNi];
  float Mh[kBjMaxNi * kBjMaxNi * kBjMaxNi], Ml[kBjMaxNi * kBjMaxNi * kBjMaxNi];
};
constexpr size_t kBjQualOffset = (sizeof(BjTab) + 255) / 256 * 256;

// (h, l) renormalised so that |l| <= ulp(h) / 2 (Fast2Sum).
__device__ __forceinline__ FF ff_norm(FF a) {
  const float h = a.hi + a.lo;
  return FF{h, a.lo - (h - a.hi)};
}

// Eigen-decomposition of a symmetric n x n matrix A (row-major, destroyed) by
// cyclic Jacobi rotations: A = Q diag(lam) Q^T, Q[m * n + a] = component m of
// eigenvector a.
inline void sym_eig(int n, double *A, double *Q, double *lam) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Q[i * n + j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) /
                         (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // Q <- Q J
          const double qkp = Q[k * n + p], qkq = Q[k * n + q];
          Q[k * n + p] = c * qkp - s * qkq;
          Q[k * n + q] = s * qkp + c * qkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

// qual[e] = 1 when every interior node of element e is unmasked and has no
// other copy (valence 1): only then is the element's interior block a
// diagonal block of A.
__global__ void k_bj_qualify(int64_t E, int64_t NG, int N, const int32_t *__restrict__ ids,
                             const int32_t *__restrict__ row_starts, uint8_t *__restrict__ qual) {
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += nth) {
    uint8_t ok = 1;
    for (int k = 1; k < N && ok; ++k)
      for (int j = 1; j < N && ok; ++j)
        for (int i = 1; i < N && ok; ++i) {
          const int32_t g = ids[e * Np + i + Nq * (j + Nq * k)];
          if (!chk(bs_pred_map_entry(g, NG), BS_CHK_PREC_ENTRY)) {
            ok = 0;
            break;
          }
          ok = g >= 0 && row_starts[g + 1] - row_starts[g] == 1;
        }
    qual[e] = ok;
  }
}

// The preconditioner's interior part, after z = D^-1 r has been written
// everywhere: z_I = A_II^-1 r_I on every qualifying element, and the r.z
// correction sum r_I (z_I - D_I^-1 r_I).  The last block adds it to the
// Jacobi part of r.z (held in st) and, except at init, forms beta and
// advances the iteration.  EPB elements per block of 256 threads, one
// thread per interior node (two when ni^3 > 256).
template <int NI>
__global__ void __launch_bounds__(256)
    k_bj_apply(int64_t E, int64_t NG, int N, const int32_t *__restrict__ ids,
               const uint8_t *__restrict__ qual, const double *__restrict__ coef, double g,
               double mlam, const BjTab *__restrict__ tab, const double *__restrict__ r,
               const double *__restrict__ dinv, double *__restrict__ z, double *partials,
               unsigned int *counter, CgState *st, int init) {
  constexpr int NN = NI * NI * NI;
  constexpr int EPB = NN >= 256 ? 1 : 256 / NN;
  constexpr int PER = (NN + 255) / 256;
  // float pairs as float2 (hi, lo): one 8-byte shared access per value
  __shared__ float2 s_a[EPB * NN], s_b[EPB * NN];
  __shared__ float2 s_V[NI * NI];
  __shared__ float s_ch[EPB], s_cl[EPB];
  if (!init && cg_halted(st)) return;
  for (int t = threadIdx.x; t < NI * NI; t += 256) {
    s_V[t] = make_float2(tab->Vh[t], tab->Vl[t]);
  }
  // a power of two bringing the residual's RMS near 1, when it lies far from it
  const double rr = init ? st->rr : st->rr_next;
  int k = 0;
  if (rr > 0.0 && isfinite(rr) && NG > 0) {
    const int e = ilogb(rr / (double)NG) / 2;
    if (e > 120 || e < -120) k = e;
  }
  const double down = ldexp(1.0, -k), up = ldexp(1.0, k);
  const FF ml = ff_split(mlam);
  const int Nq = N + 1, Np = Nq * Nq * Nq;
  double acc = 0.0;
  // Pipelined loads: while a group of elements is transformed, the r and D^-1
  // values and the coefficients of the next group and the map entries and
  // qualification flags of the group after it are in flight, so that a group
  // waits for no memory access of its own.
  int32_t nid[PER];  // map entries, two groups ahead
  uint8_t nq[PER];
  auto load_ids = [&](int64_t e0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int f = threadIdx.x + 256 * u, slot = f / NN, q = f - slot * NN;
      const int64_t e = e0 + slot;
      const bool valid = f < EPB * NN && e < E;
      const int a = q % NI, b = (q / NI) % NI, c = q / (NI * NI);
      nid[u] = valid ? ids[e * Np + (a + 1) + Nq * ((b + 1) + Nq * (c + 1))] : -1;
      if (!chk(bs_pred_map_entry(nid[u], NG), BS_CHK_PREC_ENTRY)) nid[u] = -1;
      nq[u] = valid ? qual[e] : 0;
    }
  };
  int32_t vgid[PER];  // the next group: global node (-1: not transformed), r, D^-1
  double vr[PER], vd[PER], vc = 1.0;
  auto load_vals = [&](int64_t e0) {  // from nid / nq, the map entries of group e0
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      vgid[u] = nq[u] && nid[u] >= 0 ? nid[u] : -1;
      vr[u] = vgid[u] >= 0 ? r[vgid[u]] : 0.0;
      vd[u] = vgid[u] >= 0 ? dinv[vgid[u]] : 0.0;
    }
    if (threadIdx.x < EPB) {
      const int64_t e = e0 + threadIdx.x;
      vc = coef && e < E ? coef[e] : 1.0;
    }
  };
  const int64_t gstep = (int64_t)gridDim.x * EPB, first = (int64_t)blockIdx.x * EPB;
  load_ids(first);
  load_vals(first);
  if (first + gstep < E) load_ids(first + gstep);
  for (int64_t e0 = first; e0 < E; e0 += gstep) {
    int32_t gid[PER];
    double rv[PER], dv[PER];
    bool on[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      gid[u] = vgid[u];
      on[u] = gid[u] >= 0;
      rv[u] = vr[u];
      dv[u] = vd[u];
    }
    const double cv = vc;
    if (e0 + gstep < E) {
      load_vals(e0 + gstep);
      if (e0 + 2 * gstep < E) load_ids(e0 + 2 * gstep);
    }
    if (threadIdx.x < EPB) {
      const FF c = ff_split(cv * g);
      s_ch[threadIdx.x] = c.hi;
      s_cl[threadIdx.x] = c.lo;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int f = threadIdx.x + 256 * u;
      const FF x = on[u] ? ff_split(k ? rv[u] * down : rv[u]) : FF{0.f, 0.f};
      if (f < EPB * NN) {
        s_a[f] = make_float2(x.hi, x.lo);
      }
    }
    __syncthreads();
    // (V x V x V)^T along a, b, c; the scaling; V x V x V along a, b, c.
    // Buffers alternate a -> b -> a ...; after six passes the result is in a.
#pragma unroll
    for (int pass = 0; pass < 6; ++pass) {
      const float2 *in = (pass & 1) ? s_b : s_a;
      float2 *out = (pass & 1) ? s_a : s_b;
      const int dim = pass % 3;
      const bool fwd = pass < 3;
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int f = threadIdx.x + 256 * u;
        if (f < EPB * NN) {
          const int slot = f / NN, q = f - slot * NN;
          const int ix = dim == 0 ? q % NI : (dim == 1 ? (q / NI) % NI : q / (NI * NI));
          const int stride = dim == 0 ? 1 : (dim == 1 ? NI : NI * NI);
          const int base = slot * NN + (q - ix * stride);
          FF s{0.f, 0.f};
#pragma unroll
          for (int m = 0; m < NI; ++m) {
            const int v = fwd ? m * NI + ix : ix * NI + m;
            const float2 vv = s_V[v], xv = in[base + m * stride];
            ff_fma(s, vv.x, vv.y, xv.x, xv.y);
          }
          s = ff_norm(s);
          if (pass == 2) {  // divide by d = c_e (h/2)(mu_a + mu_b + mu_c) + lambda (h/2)^3
            FF d = ml;
            ff_fma(d, s_ch[slot], s_cl[slot], __ldg(tab->Mh + q), __ldg(tab->Ml + q));
            d = ff_norm(d);
            const float x0 = 1.0f / d.hi;  // 1/d = x0 (1 + err), err from d x0 exactly
            const float p = d.hi * x0;
            const float err = ((1.0f - p) - fmaf(d.hi, x0, -p)) - d.lo * x0;
            FF o{0.f, 0.f};
            ff_fma(o, s.hi, s.lo, x0, x0 * err);
            s = ff_norm(o);
          }
          out[f] = make_float2(s.hi, s.lo);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      if (!on[u]) continue;
      const int f = threadIdx.x + 256 * u;
      const float2 zf = s_a[f];
      double zv = ff_widen(zf.x) + ff_widen(zf.y);
      if (k) zv = zv * up;
      z[gid[u]] = zv;
      acc = fma(rv[u], fma(-dv[u], rv[u], zv), acc);
    }
    __syncthreads();
  }
  const double part = block_sum<256>(acc);
  double delta;
  if (grid_combine<256>(part, partials, counter, &delta) && threadIdx.x == 0) {
    if (init) {
      st->rz = st->rz + delta;
    } else {
      const double rz = st->rz_next + delta;
      const double beta = rz / st->rz;
      st->rz = rz;
      cg_advance(st, st->rr_next, beta);
    }
  }
}

// Device tables (V and the eigenvalue sums, as float pairs) and per-element
// flags of a problem, built on first use.
inline int bj_ensure(bs_problem *P, cudaStream_t s) {
  if (P->d_bj) return BS_OK;
  const int N = P->N, Nq = N + 1, ni = N - 1;
  OpTab<double> tab;
  BS_CUDA_TRY(cudaMemcpy(&tab, P->d_tab, sizeof(tab), cudaMemcpyDeviceToHost));
  // B = W_ii^-1/2 K_ii W_ii^-1/2 = Q diag(mu) Q^T; V = W_ii^-1/2 Q
  std::vector<double> B((size_t)ni * ni), Q((size_t)ni * ni), mu(ni);
  for (int a = 0; a < ni; ++a)
    for (int b = 0; b < ni; ++b)
      B[(size_t)a * ni + b] = tab.K[(a + 1) * Nq + (b + 1)] /
                              std::sqrt(tab.w[a + 1] * tab.w[b + 1]);
  sym_eig(ni, B.data(), Q.data(), mu.data());
  BjTab h{};
  auto split = [](double v, float *hi, float *lo) {
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
  };
  for (int m = 0; m < ni; ++m)
    for (int a = 0; a < ni; ++a)
      split(Q[(size_t)m * ni + a] / std::sqrt(tab.w[m + 1]), &h.Vh[m * ni + a],
            &h.Vl[m * ni + a]);
  for (int c = 0; c < ni; ++c)
    for (int b = 0; b < ni; ++b)
      for (int a = 0; a < ni; ++a) {
        const int q = a + ni * (b + ni * c);
        split(mu[a] + mu[b] + mu[c], &h.Mh[q], &h.Ml[q]);
      }
  const int64_t E = P->map->E;
  void *mem = nullptr;
  BS_CUDA_TRY(cudaMalloc(&mem, kBjQualOffset + (size_t)(E > 0 ? E : 1)));
  P->d_bj = mem;
  BS_CUDA_TRY(cudaMemcpy(mem, &h, sizeof(h), cudaMemcpyHostToDevice));
  uint8_t *qual = static_cast<uint8_t *>(mem) + kBjQualOffset;
  if (E > 0) {
    k_bj_qualify<<<stream_grid(E, 1, 256, 4), 256, 0, s>>>(E, P->map->NG, N, P->map->d_ids,
                                                           P->map->d_row_starts, qual);
    BS_LAUNCH_CHECK();
  }
  return BS_OK;
}

// z_I = A_II^-1 r_I on the qualifying elements (z = D^-1 r already written).
inline int bj_apply(const bs_problem *P, const double *r, const double *dinv, double *z,
                    int init, cudaStream_t s) {
  const int64_t E = P->map->E;
  if (E == 0) return BS_OK;
  const BjTab *tab = static_cast<const BjTab *>(P->d_bj);
  const uint8_t *qual = static_cast<const uint8_t *>(P->d_bj) + kBjQualOffset;
  const double g = 0.5 * P->h, mlam = P->lambda * (0.5 * P->h) * (0.5 * P->h) * (0.5 * P->h);
  auto launch = [&](auto kern, int nn) -> int {
    const int epb = nn >= 256 ? 1 : 256 / nn;
    int grid = stream_grid((E + epb - 1) / epb, 1, 1, blocks_per_sm(kern, 256));
    if (grid > kMaxPartials) grid = kMaxPartials;
    kern<<<grid, 256, 0, s>>>(E, P->map->NG, P->N, P->map->d_ids, qual, P->d_coef, g, mlam, tab,
                              r, dinv, z, P->d_partials, P->d_counter, P->d_state, init);
    BS_LAUNCH_CHECK();
    return BS_OK;
  };
  switch (P->N - 1) {
    case 1: return launch(k_bj_apply<1>, 1);
    case 2: return launch(k_bj_apply<2>, 8);
    case 3: return launch(k_bj_apply<3>, 27);
    case 4: return launch(k_bj_apply<4>, 64);
    case 5: return launch(k_bj_apply<5>, 125);
    case 6: return launch(k_bj_apply<6>, 216);
    case 7: return launch(k_bj_apply<7>, 343);
    case 8: return launch(k_bj_apply<8>, 512);
    default: return fail(BS_ERR_ARG, "block Jacobi: degree %d outside 2..9", P->N);
  }
}

}  // namespace bs
