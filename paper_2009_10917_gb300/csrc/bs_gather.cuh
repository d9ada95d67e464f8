// bs_gather.cuh -- BS6 gather q_G = Z^T q_L (Table 1; Listing 4).
//
// The CSR of Z^T (rowStarts, colIds ascending within a row) makes every
// global value a short serial sum in ascending local order, so the result is
// bitwise reproducible without atomics.  Rows are cut into tiles of at most
// kTileNnz CSR entries and kTileRows rows (the paper's blockStarts, Sec. 5),
// with each tile's first row and first CSR entry precomputed.  As in
// Listing 4, a block stages a tile's values q_L[colIds[k]] in shared memory
// -- coalesced colIds reads, then kTileNnz / blockDim independent indexed
// loads per thread in flight -- and each thread then sums its rows serially
// from shared memory and writes q_G coalesced.  Each q_L value is read
// exactly once.  An optional fused epilogue forms sum_g w[g] * q_G[g] (the
// p.Ap of CG) in the same pass.
//
// Measured alternatives that were slower on GB300 (N=7, 48^3, permuted
// elements): one thread per row (51% of HBM peak), cp.async double buffering
// (54%), tiles per warp (61%), row starts staged in shared memory (57%),
// register prefetch of the next tile (66%); this form reaches about 70%.
// Later measurements: tiles of 1024 to 16384 entries, row starts or the next
// tile's indices held in registers, two tiles interleaved per block, and
// contiguous tile ranges per block were none more than 3% faster (several
// much slower); an unpermuted element order runs no faster (locality is not
// the limit: ncu shows full occupancy, DRAM bytes at the algorithmic count
// and warps waiting on the dependent colIds -> q_L loads).  Loading q_L
// through the read-only data path (__ldg) instead of as streaming loads gave
// 6%, probably because an element row read by two neighbouring tiles of the
// same wave then stays in L1.
#pragma once

#include "bs_gs.cuh"

namespace bs {

constexpr int kGatherBlock = 256;
constexpr int kTileNnz = 2048;   // CSR entries staged per tile
constexpr int kTileRows = 4096;  // rows per tile at most

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

// No-op epilogue for a gather without a fused reduction.
struct EpNone {
  __device__ __forceinline__ void operator()(double) const {}
};

// One tile [lo, hi) of rows: qG[g] = sum over k in [rowStarts[r],
// rowStarts[r+1]) of qL[colIds[k]], serially from +0 in ascending k, with
// g = rows[r] when a row list is given (the shared rows of the fused
// operator), else g = r; DOT adds w[g] * qG[g] into acc.  A block of
// kGatherBlock threads calls it together (block barriers inside); s_v holds
// kTileNnz values.
template <typename T, bool DOT, bool ROWMAP>
__device__ __forceinline__ void gather_tile(int2 lo, int2 hi,
                                            const int32_t *__restrict__ row_starts,
                                            const int32_t *__restrict__ col_ids,
                                            const int32_t *__restrict__ rows,
                                            const T *__restrict__ qL, T *__restrict__ qG,
                                            const T *__restrict__ w, T *s_v, Acc<T> &acc) {
  constexpr int U = kTileNnz / kGatherBlock;  // values per thread per tile
  {
    const int32_t r0 = lo.x, r1 = hi.x, k0 = lo.y, nk = hi.y - lo.y;
    if (nk <= kTileNnz) {
      int32_t c[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kk = threadIdx.x + u * kGatherBlock;
        c[u] = kk < nk ? __ldcs(col_ids + k0 + kk) : -1;
      }
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = c[u] >= 0 ? __ldg(qL + c[u]) : T(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kk = threadIdx.x + u * kGatherBlock;
        if (kk < nk) s_v[kk] = v[u];
      }
      __syncthreads();
      for (int32_t r = r0 + threadIdx.x; r < r1; r += kGatherBlock) {
        const T s = row_sum(s_v, row_starts[r] - k0, row_starts[r + 1] - k0);
        const int32_t g = ROWMAP ? __ldcs(rows + r) : r;
        __stcs(qG + g, s);
        if (DOT) acc.add(__ldcs(w + g), s);
      }
      __syncthreads();
    } else {  // a single row longer than a tile: read straight from memory
      for (int32_t r = r0 + threadIdx.x; r < r1; r += kGatherBlock) {
        const int32_t a = row_starts[r], b = row_starts[r + 1];
        T s = T(0);
        if (a < b) s = plus_zero(qL[col_ids[a]]);
        for (int32_t k = a + 1; k < b; ++k) s = s + qL[col_ids[k]];
        const int32_t g = ROWMAP ? rows[r] : r;
        qG[g] = s;
        if (DOT) acc.add(w[g], s);
      }
    }
  }
}

// The whole gather, tiles in grid-stride order.  DOT: also reduce
// sum_g w[g] * qG[g], plus the nextra per-block partials in extra (the fused
// operator's own terms, summed after the gather's in index order), into ep().
template <typename T, bool DOT, bool ROWMAP, class Ep>
__global__ void __launch_bounds__(kGatherBlock)
    k_gather(int64_t ntiles, const int2 *__restrict__ tiles,
             const int32_t *__restrict__ row_starts, const int32_t *__restrict__ col_ids,
             const int32_t *__restrict__ rows, const T *__restrict__ qL, T *__restrict__ qG,
             const T *__restrict__ w, double *partials, unsigned int *counter,
             const double *__restrict__ extra, int64_t nextra, Ep ep, const CgState *st) {
  __shared__ T s_v[kTileNnz];
  if (cg_halted(st)) return;
  Acc<T> acc;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
    gather_tile<T, DOT, ROWMAP>(tiles[t], tiles[t + 1], row_starts, col_ids, rows, qL, qG, w,
                                s_v, acc);
  if (DOT) {
    const double part = block_sum<kGatherBlock>(acc.value());
    double total;
    if (grid_combine<kGatherBlock>(part, partials, counter, &total)) {
      if (nextra == 0) {
        if (threadIdx.x == 0) ep(total);
      } else {
        double v = 0.0;
        for (int64_t b = threadIdx.x; b < nextra; b += kGatherBlock) v = v + __ldcg(extra + b);
        v = block_sum<kGatherBlock>(v);
        if (threadIdx.x == 0) ep(total + v);
      }
    }
  }
}

// The gather of every row (rows == false) or of the fused operator's shared
// rows (rows == true), with the optional fused reduction.
template <typename T, bool DOT, class Ep>
int launch_gather_rows(const bs_map *m, bool shared, const T *qL, T *qG, const T *w,
                       double *partials, unsigned int *counter, const double *extra,
                       int64_t nextra, Ep ep, const CgState *st, cudaStream_t s) {
  const int64_t nt = shared ? m->nsh_tiles : m->ntiles;
  auto launch = [&](auto kern) -> int {
    int grid = stream_grid(nt, 1, 1, blocks_per_sm(kern, kGatherBlock));
    if (grid < 1) return fail(BS_ERR_CUDA, "no device");
    if (DOT && grid > kMaxPartials) grid = kMaxPartials;
    if (shared)
      kern<<<grid, kGatherBlock, 0, s>>>(nt, m->d_sh_tiles, m->d_sh_starts, m->d_sh_cols,
                                         m->d_sh_rows, qL, qG, w, partials, counter, extra,
                                         nextra, ep, st);
    else
      kern<<<grid, kGatherBlock, 0, s>>>(nt, m->d_tiles, m->d_row_starts, m->d_col_ids,
                                         nullptr, qL, qG, w, partials, counter, extra, nextra,
                                         ep, st);
    BS_LAUNCH_CHECK();
    return BS_OK;
  };
  return shared ? launch(k_gather<T, DOT, true, Ep>) : launch(k_gather<T, DOT, false, Ep>);
}

template <typename T, bool DOT, class Ep>
int launch_gather(const bs_map *m, const T *qL, T *qG, const T *w, double *partials,
                  unsigned int *counter, Ep ep, const CgState *st, cudaStream_t s) {
  return launch_gather_rows<T, DOT, Ep>(m, false, qL, qG, w, partials, counter, nullptr, 0, ep,
                                        st, s);
}

}  // namespace bs
