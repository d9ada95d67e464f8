// bs_gs.cuh -- BS6 gather and BS7 scatter kernels (Table 1; Listings 4-5).
//
// Scatter: one thread per four consecutive local nodes -- a 128-bit load of
// the int32 map, four indexed loads of q_G (L2 serves the repeats of shared
// nodes), two 128-bit streaming stores when none of the four is masked.
//
// Gather: the CSR of Z^T (rowStarts, colIds ascending within a row) makes
// every global value a short serial sum in ascending local order, so the
// result is bitwise reproducible without atomics.  One thread per global
// row; rows of a warp are consecutive, so rowStarts/colIds reads coalesce
// and each q_L value is read exactly once.  An optional fused epilogue forms
// sum_g w[g] * q_G[g] (the p.Ap of CG) in the same pass.
#pragma once

#include "bs_stream.cuh"

struct bs_map {
  int device;
  int32_t E, N;
  int64_t NL, NG, nnz;
  int32_t *d_ids;         // [NL] local -> global, < 0 masked
  int32_t *d_row_starts;  // [NG + 1]
  int32_t *d_col_ids;     // [nnz], ascending within each row
};

namespace bs {

template <typename T> struct Vec2Of;
template <> struct Vec2Of<double> { using type = double2; };
template <> struct Vec2Of<float> { using type = float2; };

// qL[l] = qG[ids[l]] for ids[l] >= 0.  VEC: qL is 16-byte aligned (double)
// or 8-byte aligned (float), so pairs of outputs go out as one store.
template <typename T, bool VEC>
__global__ void __launch_bounds__(kStreamBlock)
    k_scatter(int64_t NL, const int32_t *__restrict__ ids, const T *__restrict__ qG,
              T *__restrict__ qL) {
  using V2 = typename Vec2Of<T>::type;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = NL / 4;
  const int4 *ids4 = reinterpret_cast<const int4 *>(ids);
  for (int64_t q = tid; q < n4; q += nth) {
    const int4 id = __ldcs(ids4 + q);
    const int64_t l = q * 4;
    if (VEC && (id.x | id.y | id.z | id.w) >= 0) {
      V2 a, b;
      a.x = qG[id.x];
      a.y = qG[id.y];
      b.x = qG[id.z];
      b.y = qG[id.w];
      V2 *o = reinterpret_cast<V2 *>(qL + l);
      __stcs(o, a);
      __stcs(o + 1, b);
    } else {
      if (id.x >= 0) qL[l] = qG[id.x];
      if (id.y >= 0) qL[l + 1] = qG[id.y];
      if (id.z >= 0) qL[l + 2] = qG[id.z];
      if (id.w >= 0) qL[l + 3] = qG[id.w];
    }
  }
  for (int64_t l = n4 * 4 + tid; l < NL; l += nth) {
    const int32_t id = ids[l];
    if (id >= 0) qL[l] = qG[id];
  }
}

template <typename T>
int launch_scatter(const bs_map *m, const T *qG, T *qL, cudaStream_t s) {
  const bool vec = (reinterpret_cast<uintptr_t>(qL) % (2 * sizeof(T))) == 0;
  auto kern = vec ? k_scatter<T, true> : k_scatter<T, false>;
  const int64_t work = m->NL / 4 > 0 ? m->NL / 4 : m->NL;
  const int grid = stream_grid(work, 1, kStreamBlock, blocks_per_sm(kern, kStreamBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  kern<<<grid, kStreamBlock, 0, s>>>(m->NL, m->d_ids, qG, qL);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// No-op epilogue for a gather without a fused reduction.
struct EpNone {
  __device__ __forceinline__ void operator()(double) const {}
};

// qG[g] = sum over k in [rowStarts[g], rowStarts[g+1]) of qL[colIds[k]],
// serially from +0.  DOT: also reduce sum_g w[g] * qG[g] into ep().
template <typename T, bool DOT, class Ep>
__global__ void __launch_bounds__(kReduceBlock)
    k_gather(int64_t NG, const int32_t *__restrict__ row_starts,
             const int32_t *__restrict__ col_ids, const T *__restrict__ qL,
             T *__restrict__ qG, const T *__restrict__ w, double *partials,
             unsigned int *counter, Ep ep, const CgState *st) {
  if (cg_halted(st)) return;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  Acc<T> acc;
  for (int64_t g = tid; g < NG; g += nth) {
    const int32_t k0 = row_starts[g], k1 = row_starts[g + 1];
    T s = T(0);
    for (int32_t k = k0; k < k1; ++k) s = s + qL[__ldcs(col_ids + k)];
    __stcs(qG + g, s);
    if (DOT) acc.add(__ldcs(w + g), s);
  }
  if (DOT) {
    const double part = block_sum<kReduceBlock>(acc.value());
    double total;
    if (grid_combine<kReduceBlock>(part, partials, counter, &total) && threadIdx.x == 0)
      ep(total);
  }
}

template <typename T, bool DOT, class Ep>
int launch_gather(const bs_map *m, const T *qL, T *qG, const T *w, double *partials,
                  unsigned int *counter, Ep ep, const CgState *st, cudaStream_t s) {
  auto kern = k_gather<T, DOT, Ep>;
  int grid = stream_grid(m->NG, 1, kReduceBlock, blocks_per_sm(kern, kReduceBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  if (DOT && grid > kMaxPartials) grid = kMaxPartials;
  kern<<<grid, kReduceBlock, 0, s>>>(m->NG, m->d_row_starts, m->d_col_ids, qL, qG, w, partials,
                                     counter, ep, st);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

}  // namespace bs
