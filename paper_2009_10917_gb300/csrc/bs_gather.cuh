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
// same wave then stays in L1.  This staged form serves a q_L not aligned to
// two values, the fused operator's shared rows and the batched solver; the
// FP64 and FP32 gathers run the pipelined form further down (82% of the peak
// in the same setting, FP64).
#pragma once

#include "bs_gs.cuh"
#include "bs_tiles.h"

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

// Sizes the checked build tests a gather's indices against: the CSR's rows
// and entries, q_L's and q_G's lengths.
struct GBounds {
  int64_t rows, nnz, nl, ng;
};

// One tile [lo, hi) of rows: qG[g] = sum over k in [rowStarts[r],
// rowStarts[r+1]) of qL[colIds[k]], serially from +0 in ascending k, with
// g = rows[r] when a row list is given (the shared rows of the fused
// operator), else g = r; DOT adds w[g] * qG[g] into acc.  A block of
// kGatherBlock threads calls it together (block barriers inside); s_v holds
// kTileNnz values; gb bounds the indices in the checked build.
template <typename T, bool DOT, bool ROWMAP>
__device__ __forceinline__ void gather_tile(int2 lo, int2 hi,
                                            const int32_t *__restrict__ row_starts,
                                            const int32_t *__restrict__ col_ids,
                                            const int32_t *__restrict__ rows,
                                            const T *__restrict__ qL, T *__restrict__ qG,
                                            const T *__restrict__ w, T *s_v, Acc<T> &acc,
                                            const GBounds &gb) {
  constexpr int U = kTileNnz / kGatherBlock;  // values per thread per tile
  if (!chk(bs_pred_tile(lo.x, hi.x, lo.y, hi.y, gb.rows, gb.nnz, kTileNnz), BS_CHK_GATHER_TILE))
    return;  // block-uniform: every thread skips the tile and its barriers
  {
    const int32_t r0 = lo.x, r1 = hi.x, k0 = lo.y, nk = hi.y - lo.y;
    if (nk <= kTileNnz) {
      int32_t c[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kk = threadIdx.x + u * kGatherBlock;
        c[u] = kk < nk ? __ldcs(col_ids + k0 + kk) : -1;
        if (!chk(c[u] < 0 || bs_pred_index(c[u], gb.nl), BS_CHK_GATHER_COL)) c[u] = -1;
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
        int a = row_starts[r] - k0, b = row_starts[r + 1] - k0;
        if (!chk(bs_pred_row(a, b, nk), BS_CHK_GATHER_ROW)) a = b = 0;
        const T s = row_sum(s_v, a, b);
        const int32_t g = ROWMAP ? __ldcs(rows + r) : r;
        if (!chk(bs_pred_index(g, gb.ng), BS_CHK_GATHER_ROW)) continue;
        __stcs(qG + g, s);
        if (DOT) acc.add(__ldcs(w + g), s);
      }
      __syncthreads();
    } else {  // a single row longer than a tile: read straight from memory
      for (int32_t r = r0 + threadIdx.x; r < r1; r += kGatherBlock) {
        int32_t a = row_starts[r], b = row_starts[r + 1];
        if (!chk(bs_pred_row(a, b, gb.nnz), BS_CHK_GATHER_ROW)) a = b = 0;
        T s = T(0);
        if (a < b) {
          const int32_t c = col_ids[a];
          if (chk(bs_pred_index(c, gb.nl), BS_CHK_GATHER_COL)) s = plus_zero(qL[c]);
        }
        for (int32_t k = a + 1; k < b; ++k) {
          const int32_t c = col_ids[k];
          if (chk(bs_pred_index(c, gb.nl), BS_CHK_GATHER_COL)) s = s + qL[c];
        }
        const int32_t g = ROWMAP ? rows[r] : r;
        if (!chk(bs_pred_index(g, gb.ng), BS_CHK_GATHER_ROW)) continue;
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
             const double *__restrict__ extra, int64_t nextra, Ep ep, const CgState *st,
             GBounds gb) {
  __shared__ T s_v[kTileNnz];
  if (cg_halted(st)) return;
  Acc<T> acc;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
    gather_tile<T, DOT, ROWMAP>(tiles[t], tiles[t + 1], row_starts, col_ids, rows, qL, qG, w,
                                s_v, acc, gb);
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

// ------------------------------------------------------------ pipelined gather (FP64, FP32)
//
// The staged-tile gather above waits, tile after tile, on two dependent
// loads (colIds, then q_L).  This form hides them: the map is re-encoded once
// per tile as the distinct chunks of q_L the tile reads (two values each:
// 16 bytes in FP64, 8 in FP32, one encoding for both) and a blob of uint16
// entry offsets into those chunks plus uint16 row starts.  A block copies tile t + 1's chunks and blob into shared memory with
// cp.async while it sums tile t (two stages), and loads tile t + 2's chunk
// ids into registers meanwhile, so every global load it waits for was issued
// a tile earlier.  Sums run over the same entries in the same order as the
// CSR: the result is bitwise the staged-tile gather's.  A row longer than a
// tile gets a tile of its own, summed straight from the CSR.  The blob also
// lists the tile's rows by length (longest first): thread p sums row ord[p],
// so the 32 rows of a warp have about equal lengths.  In CSR order a warp
// waited on its longest row, issuing about three times the dependent FP64
// adds the rows need on GB300's narrow FP64 pipe (3.5% faster in the lab).
// Tiles of 1024 entries for 256-thread blocks (27 KB of shared memory, eight
// blocks per SM) ran 1% faster than 2048 for 512 threads; three stages, or
// 128-thread blocks, were slower.
// tile sizes kAgChunks, kAgEntries, kAgRows and kAgBlob16: bs_tiles.h
constexpr int kAgBlock = 256;
// One stage: the tile's chunks (two values of T each), then its blob.  The
// FP32 gather uses the same encoding with 8-byte chunks.
template <typename T>
constexpr int ag_stage() {
  return kAgChunks * 2 * (int)sizeof(T) + kAgBlob16 * 16;
}
template <typename T>
constexpr int ag_smem() {
  return 2 * ag_stage<T>();
}

__device__ __forceinline__ void ag_cp16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void ag_cp8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void ag_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void ag_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T, bool DOT, class Ep>
__global__ void __launch_bounds__(kAgBlock)
    k_gather_async(int64_t ntiles, const int4 *__restrict__ info,
                   const int32_t *__restrict__ chunks, const uint4 *__restrict__ blob,
                   const int32_t *__restrict__ row_starts, const int32_t *__restrict__ col_ids,
                   const T *__restrict__ qL, T *__restrict__ qG, const T *__restrict__ w,
                   double *partials, unsigned int *counter, Ep ep, const CgState *st,
                   GBounds gb) {
  constexpr int kStage = ag_stage<T>(), kChunkBytes = 2 * (int)sizeof(T);
  extern __shared__ __align__(16) unsigned char ag_sm[];
  constexpr int CPT = (kAgChunks + kAgBlock - 1) / kAgBlock;  // chunk ids per thread
  if (cg_halted(st)) return;
  // checked build: the end of the chunk and blob arrays, for the tile tests
  const int4 ag_end = BS_CHECK ? info[ntiles] : make_int4(0, 0, 0, 0);
  auto chunks_ok = [&](int c0, int c1) {
    return chk(c0 >= 0 && c0 <= c1 && c1 - c0 <= kAgChunks && c1 <= ag_end.y,
               BS_CHK_GATHER_TILE);
  };
  const int64_t G = gridDim.x;
  int64_t t = blockIdx.x;
  int idsA[CPT], idsB[CPT];
  auto load_ids = [&](int64_t tt, int *ids) {
#pragma unroll
    for (int u = 0; u < CPT; ++u) ids[u] = -1;
    if (tt >= ntiles) return;
    const int4 a = info[tt];
    if (a.w < 0) return;
    const int c0 = a.y, c1 = info[tt + 1].y;
    if (!chunks_ok(c0, c1)) return;
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int i = threadIdx.x + u * kAgBlock;
      ids[u] = i < c1 - c0 ? __ldcs(chunks + c0 + i) : -1;
      if (ids[u] >= 0 && !chk(bs_pred_index(ids[u], gb.nl / 2), BS_CHK_GATHER_CHUNK)) ids[u] = -1;
    }
  };
  auto issue = [&](int64_t tt, const int *ids, int stage) {
    if (tt < ntiles) {
      const int4 a = info[tt];
      if (a.w >= 0) {
        unsigned char *base = ag_sm + stage * kStage;
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
          if (ids[u] < 0) continue;
          unsigned char *dst = base + (threadIdx.x + u * kAgBlock) * kChunkBytes;
          if constexpr (sizeof(T) == 8)
            ag_cp16(dst, qL + 2ll * ids[u]);
          else
            ag_cp8(dst, qL + 2ll * ids[u]);
        }
        const int b0 = a.z, b1 = info[tt + 1].z;
        if (chk(b0 >= 0 && b0 <= b1 && b1 - b0 <= kAgBlob16 && b1 <= ag_end.z,
                BS_CHK_GATHER_TILE))
          for (int i = threadIdx.x; i < b1 - b0; i += kAgBlock)
            ag_cp16(base + kAgChunks * kChunkBytes + i * 16, blob + b0 + i);
      }
    }
    ag_commit();
  };
  Acc<T> acc;
  load_ids(t, idsA);
  load_ids(t + G, idsB);
  issue(t, idsA, 0);
  int stage = 0;
  for (; t < ntiles; t += G) {
    load_ids(t + 2 * G, idsA);  // idsA is free again: tile t's copies are issued
    issue(t + G, idsB, stage ^ 1);
    ag_wait<1>();  // tile t's copies have landed (only tile t + 1's may be pending)
    __syncthreads();
    const int4 a = info[t];
    const int r0 = a.x;
    if (a.w >= 0) {
      const unsigned char *base = ag_sm + stage * kStage;
      const T *qv = reinterpret_cast<const T *>(base);
      const unsigned short *off =
          reinterpret_cast<const unsigned short *>(base + kAgChunks * kChunkBytes);
      int ne = a.w >> 16, rows = a.w & 0xffff;
      const int nst = 2 * (info[t + 1].y - a.y);  // staged values
      if (!chk(ne <= kAgEntries && rows <= kAgRows && r0 >= 0 && r0 + rows <= gb.ng &&
                   chunks_ok(a.y, info[t + 1].y),
               BS_CHK_GATHER_TILE))
        ne = rows = 0;
      const unsigned short *rstart = off + ((ne + 7) & ~7);
      const unsigned short *ord = rstart + ((rows + 1 + 7) & ~7);
      for (int p = threadIdx.x; p < rows; p += kAgBlock) {
        int r = ord[p];
        if (!chk(bs_pred_index(r, rows), BS_CHK_GATHER_STAGED)) continue;
        int b0 = rstart[r], b1 = rstart[r + 1];
        if (!chk(bs_pred_row(b0, b1, ne), BS_CHK_GATHER_STAGED)) b0 = b1 = 0;
        T s = T(0);
        if (b0 < b1) {
          const int o = off[b0];
          if (chk(bs_pred_staged(o, nst), BS_CHK_GATHER_STAGED)) s = plus_zero(qv[o]);
          for (int k = b0 + 1; k < b1; ++k) {
            const int ok = off[k];
            if (chk(bs_pred_staged(ok, nst), BS_CHK_GATHER_STAGED)) s = s + qv[ok];
          }
        }
        __stcs(qG + r0 + r, s);
        if (DOT) acc.add(__ldcs(w + r0 + r), s);
      }
    } else {  // rows longer than a tile: straight from the CSR
      int r1 = info[t + 1].x;
      if (!chk(r0 >= 0 && r0 <= r1 && r1 <= gb.ng, BS_CHK_GATHER_TILE)) r1 = r0;
      for (int r = r0 + threadIdx.x; r < r1; r += kAgBlock) {
        int32_t b0 = row_starts[r], b1 = row_starts[r + 1];
        if (!chk(bs_pred_row(b0, b1, gb.nnz), BS_CHK_GATHER_ROW)) b0 = b1 = 0;
        T s = T(0);
        if (b0 < b1) {
          const int32_t c = col_ids[b0];
          if (chk(bs_pred_index(c, gb.nl), BS_CHK_GATHER_COL)) s = plus_zero(qL[c]);
        }
        for (int32_t k = b0 + 1; k < b1; ++k) {
          const int32_t c = col_ids[k];
          if (chk(bs_pred_index(c, gb.nl), BS_CHK_GATHER_COL)) s = s + qL[c];
        }
        qG[r] = s;
        if (DOT) acc.add(w[r], s);
      }
    }
    __syncthreads();  // stage is refilled by the next iteration's issue
#pragma unroll
    for (int u = 0; u < CPT; ++u) idsB[u] = idsA[u];
    stage ^= 1;
  }
  ag_wait<0>();
  if (DOT) {
    const double part = block_sum<kAgBlock>(acc.value());
    double total;
    if (grid_combine<kAgBlock>(part, partials, counter, &total) && threadIdx.x == 0) ep(total);
  }
}

template <typename T, bool DOT, class Ep>
int launch_gather_async(const bs_map *m, const T *qL, T *qG, const T *w, double *partials,
                        unsigned int *counter, Ep ep, const CgState *st, cudaStream_t s) {
  auto kern = k_gather_async<T, DOT, Ep>;
  constexpr int smem = ag_smem<T>();
  const int bps = occupancy_blocks_smem((const void *)kern, kAgBlock, smem);
  if (bps < 1) return fail(BS_ERR_CUDA, "pipelined gather: %d B of shared memory refused", smem);
  int grid = stream_grid(m->ag_ntiles, 1, 1, bps);
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  if (DOT && grid > kMaxPartials) grid = kMaxPartials;
  kern<<<grid, kAgBlock, smem, s>>>(m->ag_ntiles, m->d_ag_info, m->d_ag_chunks, m->d_ag_blob,
                                    m->d_row_starts, m->d_col_ids, qL, qG, w, partials, counter,
                                    ep, st, GBounds{m->NG, m->nnz, m->NL, m->NG});
  BS_LAUNCH_CHECK();
  return BS_OK;
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
                                         nextra, ep, st,
                                         GBounds{m->nsh, m->nnz_sh, m->NL, m->NG});
    else
      kern<<<grid, kGatherBlock, 0, s>>>(nt, m->d_tiles, m->d_row_starts, m->d_col_ids,
                                         nullptr, qL, qG, w, partials, counter, extra, nextra,
                                         ep, st, GBounds{m->NG, m->nnz, m->NL, m->NG});
    BS_LAUNCH_CHECK();
    return BS_OK;
  };
  return shared ? launch(k_gather<T, DOT, true, Ep>) : launch(k_gather<T, DOT, false, Ep>);
}

template <typename T, bool DOT, class Ep>
int launch_gather(const bs_map *m, const T *qL, T *qG, const T *w, double *partials,
                  unsigned int *counter, Ep ep, const CgState *st, cudaStream_t s) {
  // the pipelined form copies two values per chunk: q_L aligned to 2 sizeof(T)
  if (m->d_ag_info && ((uintptr_t)qL % (2 * sizeof(T))) == 0)
    return launch_gather_async<T, DOT, Ep>(m, qL, qG, w, partials, counter, ep, st, s);
  return launch_gather_rows<T, DOT, Ep>(m, false, qL, qG, w, partials, counter, nullptr, 0, ep,
                                        st, s);
}

}  // namespace bs
