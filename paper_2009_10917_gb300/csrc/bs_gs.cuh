// bs_gs.cuh -- BS6 gather and BS7 scatter kernels (Table 1; Listings 4-5).
//
// Scatter: elements are visited in the order of their smallest global index
// (sorted once when the map is built, from the map alone), so elements that
// share global nodes run close together in time and the repeated q_G reads
// hit L2 instead of HBM.  A block covers max(1, 256 / Np) elements at a
// time, one thread per local node (coalesced map loads and q_L stores), and
// U such element groups per sweep, so U value loads per thread are in
// flight.
//
// Gather: the CSR of Z^T (rowStarts, colIds ascending within a row) makes
// every global value a short serial sum in ascending local order, so the
// result is bitwise reproducible without atomics.  Rows are cut into tiles
// of at most kTileNnz CSR entries and kTileRows rows (the paper's
// blockStarts, Sec. 5) whose first row and first CSR entry are precomputed.
// A block loads a tile's column indices and row starts with independent
// coalesced loads, then the values q_L[colIds[k]] with independent indexed
// loads (kTileNnz / blockDim per thread), all into shared memory; each thread
// then sums its rows serially from shared memory and writes q_G coalesced,
// so a tile waits on two memory latencies and nothing in the row loop
// touches global memory except the store.  Each q_L value is read exactly
// once.  An optional fused epilogue forms sum_g w[g] * q_G[g] (the p.Ap of
// CG) in the same pass.
#pragma once

#include "bs_stream.cuh"

struct bs_map {
  int device;
  int32_t E, N;
  int64_t NL, NG, nnz;
  int32_t *d_ids;         // [NL] local -> global, < 0 masked
  int32_t *d_row_starts;  // [NG + 1]
  int32_t *d_col_ids;     // [nnz], ascending within each row
  int64_t ntiles;
  int2 *d_tiles;          // [ntiles + 1] (first row, first CSR entry) per tile
  int32_t *d_elem_order;  // [E] elements by smallest global index
};

namespace bs {

template <typename T> struct Vec2Of;
template <> struct Vec2Of<double> { using type = double2; };
template <> struct Vec2Of<float> { using type = float2; };

constexpr int kScatterBlock = 256;

// qL[l] = qG[ids[l]] for ids[l] >= 0, element by element in `order`.
template <typename T, int U>
__global__ void __launch_bounds__(kScatterBlock)
    k_scatter(int64_t E, int Np, const int32_t *__restrict__ order,
              const int32_t *__restrict__ ids, const T *__restrict__ qG, T *__restrict__ qL) {
  // Np <= 256: EPB elements per group, thread -> (element slot, node) once;
  // Np > 256: one element per group, threads stride over its nodes.
  const int epb = Np <= kScatterBlock ? kScatterBlock / Np : 1;
  const int sub = Np <= kScatterBlock ? (int)threadIdx.x / Np : 0;
  const int node0 = Np <= kScatterBlock ? (int)threadIdx.x - sub * Np : (int)threadIdx.x;
  if (sub >= epb) return;
  const int64_t groups = (E + epb - 1) / epb;
  for (int node = node0; node < Np; node += kScatterBlock) {
    for (int64_t g = blockIdx.x; g < groups; g += (int64_t)U * gridDim.x) {
      int64_t l[U];
      int32_t id[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t slot = (g + (int64_t)u * gridDim.x) * epb + sub;
        l[u] = slot < E ? (int64_t)__ldg(order + slot) * Np + node : -1;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) id[u] = l[u] >= 0 ? __ldcs(ids + l[u]) : -1;
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = id[u] >= 0 ? qG[id[u]] : T(0);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (id[u] >= 0) __stcs(qL + l[u], v[u]);
    }
  }
}

template <typename T>
int launch_scatter(const bs_map *m, const T *qG, T *qL, cudaStream_t s) {
  constexpr int U = 4;
  auto kern = k_scatter<T, U>;
  const int Np = (m->N + 1) * (m->N + 1) * (m->N + 1);
  const int epb = Np <= kScatterBlock ? kScatterBlock / Np : 1;
  const int64_t groups = (m->E + epb - 1) / epb;
  int grid = stream_grid(groups, U, 1, blocks_per_sm(kern, kScatterBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  kern<<<grid, kScatterBlock, 0, s>>>(m->E, Np, m->d_elem_order, m->d_ids, qG, qL);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// No-op epilogue for a gather without a fused reduction.
struct EpNone {
  __device__ __forceinline__ void operator()(double) const {}
};

constexpr int kGatherBlock = 256;
constexpr int kTileNnz = 2048;   // CSR entries staged per tile
constexpr int kTileRows = 2048;  // rows per tile at most

// +0.0 + v without an FP64 add: v, except that -0.0 becomes +0.0.
__device__ __forceinline__ double plus_zero(double v) {
  return __double_as_longlong(v) == (long long)0x8000000000000000ull ? 0.0 : v;
}
__device__ __forceinline__ float plus_zero(float v) {
  return __float_as_uint(v) == 0x80000000u ? 0.0f : v;
}

// Serial sum of vals[a..b) in ascending order, from +0.0.
template <typename T>
__device__ __forceinline__ T row_sum(const T *vals, int a, int b) {
  if (a >= b) return T(0);
  T s = plus_zero(vals[a]);
  for (int k = a + 1; k < b; ++k) s = s + vals[k];
  return s;
}

// qG[g] = sum over k in [rowStarts[g], rowStarts[g+1]) of qL[colIds[k]],
// serially from +0 in ascending k.  DOT: also reduce sum_g w[g] * qG[g].
template <typename T, bool DOT, class Ep>
__global__ void __launch_bounds__(kGatherBlock)
    k_gather(int64_t ntiles, const int2 *__restrict__ tiles,
             const int32_t *__restrict__ row_starts, const int32_t *__restrict__ col_ids,
             const T *__restrict__ qL, T *__restrict__ qG, const T *__restrict__ w,
             double *partials, unsigned int *counter, Ep ep, const CgState *st) {
  constexpr int U = kTileNnz / kGatherBlock;   // values per thread per tile
  constexpr int R = kTileRows / kGatherBlock;  // rows per thread per tile
  __shared__ T s_v[kTileNnz];
  __shared__ int32_t s_rs[kTileRows + 1];
  if (cg_halted(st)) return;
  Acc<T> acc;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 lo = tiles[t], hi = tiles[t + 1];
    const int32_t r0 = lo.x, nr = hi.x - lo.x, k0 = lo.y, nk = hi.y - lo.y;
    if (nk <= kTileNnz) {
      int32_t c[U], rs[R];
      T wr[DOT ? R : 1];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kk = threadIdx.x + u * kGatherBlock;
        c[u] = kk < nk ? __ldcs(col_ids + k0 + kk) : -1;
      }
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int rr = threadIdx.x + q * kGatherBlock;
        rs[q] = rr < nr ? __ldcs(row_starts + r0 + rr) : 0;
        if (DOT) wr[q] = rr < nr ? __ldcs(w + r0 + rr) : T(0);
      }
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = c[u] >= 0 ? __ldcs(qL + c[u]) : T(0);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int rr = threadIdx.x + q * kGatherBlock;
        if (rr < nr) s_rs[rr] = rs[q] - k0;
      }
      if (threadIdx.x == 0) s_rs[nr] = nk;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kk = threadIdx.x + u * kGatherBlock;
        if (kk < nk) s_v[kk] = v[u];
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int rr = threadIdx.x + q * kGatherBlock;
        if (rr < nr) {
          const T s = row_sum(s_v, s_rs[rr], s_rs[rr + 1]);
          __stcs(qG + r0 + rr, s);
          if (DOT) acc.add(wr[q], s);
        }
      }
      __syncthreads();
    } else {  // a single row longer than a tile: read straight from memory
      for (int32_t r = r0 + threadIdx.x; r < hi.x; r += kGatherBlock) {
        const int32_t a = row_starts[r], b = row_starts[r + 1];
        T s = T(0);
        if (a < b) s = plus_zero(qL[col_ids[a]]);
        for (int32_t k = a + 1; k < b; ++k) s = s + qL[col_ids[k]];
        qG[r] = s;
        if (DOT) acc.add(w[r], s);
      }
    }
  }
  if (DOT) {
    const double part = block_sum<kGatherBlock>(acc.value());
    double total;
    if (grid_combine<kGatherBlock>(part, partials, counter, &total) && threadIdx.x == 0)
      ep(total);
  }
}

template <typename T, bool DOT, class Ep>
int launch_gather(const bs_map *m, const T *qL, T *qG, const T *w, double *partials,
                  unsigned int *counter, Ep ep, const CgState *st, cudaStream_t s) {
  auto kern = k_gather<T, DOT, Ep>;
  int grid = stream_grid(m->ntiles, 1, 1, blocks_per_sm(kern, kGatherBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  if (DOT && grid > kMaxPartials) grid = kMaxPartials;
  kern<<<grid, kGatherBlock, 0, s>>>(m->ntiles, m->d_tiles, m->d_row_starts, m->d_col_ids, qL,
                                     qG, w, partials, counter, ep, st);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

}  // namespace bs
