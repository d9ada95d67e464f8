// bs_gs.cuh -- the map object and the BS7 scatter kernel (Table 1; Listing 5).
//
// Scatter: elements are visited in the order of their smallest global index
// (sorted once when the map is built, from the map alone), so elements that
// share global nodes run close together in time and the repeated q_G reads
// hit L2 instead of HBM.  A block covers max(1, 256 / Np) elements at a
// time, one thread per local node (coalesced map loads and q_L stores), and
// U such element groups per sweep, so U value loads per thread are in
// flight.  When Np is even and q_L is 16-byte aligned, a thread takes two
// consecutive local nodes (one 8-byte map load, one 16-byte store) and two
// groups per sweep: measured 6.2 TB/s against 5.9 TB/s for one node per
// thread and four groups on the N = 7, 48^3 mesh.
//
// The BS6 gather kernel lives in bs_gather.cuh.
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
  // Fused operator (bs_op.cuh): the map re-encoded for an element kernel that
  // writes single-copy nodes itself, and the CSR of the shared rows alone.
  int32_t *d_ids_f;       // [NL] g if node g has != 1 copies, -2 - g if one, -1 masked
  int64_t nsh, nnz_sh, nsh_tiles;
  int32_t *d_sh_rows;     // [nsh] global index of each row with != 1 copies, ascending
  int32_t *d_sh_starts;   // [nsh + 1]
  int32_t *d_sh_cols;     // [nnz_sh] the rows' CSR entries, ascending local index
  int2 *d_sh_tiles;       // [nsh_tiles + 1]
  // The pipelined FP64 gather (bs_gather.cuh, k_gather_async): per tile the
  // distinct 16-byte chunks of q_L it reads and a blob of uint16 entry offsets,
  // row starts and summing order; NULL when N_G is 0.  With N_L odd the row
  // holding the last local node is summed from the CSR (its chunk would leave
  // q_L).
  int64_t ag_ntiles;
  int4 *d_ag_info;        // [ag_ntiles + 1] first row, first chunk, first blob word,
                          // (entries << 16 | rows), or -1: rows summed straight from the CSR
  int32_t *d_ag_chunks;   // chunk c covers q_L[2c], q_L[2c + 1]
  uint4 *d_ag_blob;       // 16-byte words
};

namespace bs {

template <typename T> struct Vec2Of;
template <> struct Vec2Of<double> { using type = double2; };
template <> struct Vec2Of<float> { using type = float2; };

constexpr int kScatterBlock = 256;

// qL[l] = qG[ids[l]] for ids[l] >= 0, element by element in `order`.  NG
// bounds the map entries in the checked build.
template <typename T, int U>
__global__ void __launch_bounds__(kScatterBlock)
    k_scatter(int64_t E, int64_t NG, int Np, const int32_t *__restrict__ order,
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
        if (l[u] >= 0 && !chk(bs_pred_index(l[u] / Np, E), BS_CHK_SCATTER_ENTRY)) l[u] = -1;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        id[u] = l[u] >= 0 ? __ldcs(ids + l[u]) : -1;
        if (!chk(bs_pred_map_entry(id[u], NG), BS_CHK_SCATTER_ENTRY)) id[u] = -1;
      }
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = id[u] >= 0 ? qG[id[u]] : T(0);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (id[u] >= 0) __stcs(qL + l[u], v[u]);
    }
  }
}

// Two consecutive local nodes per thread (Np even; q_L 16-byte aligned, so
// every element row and pair is aligned), U element groups per trip.  The
// element order and map entries of the next trip are loaded while this trip's
// q_G values are in flight, so a trip waits on one dependent load instead of
// three (order -> ids -> q_G); measured 6% faster than loading them in turn.
template <typename T, int U>
__global__ void __launch_bounds__(kScatterBlock)
    k_scatter2(int64_t E, int64_t NG, int Np, const int32_t *__restrict__ order,
               const int32_t *__restrict__ ids, const T *__restrict__ qG, T *__restrict__ qL) {
  using V2 = typename Vec2Of<T>::type;
  const int pairs = Np / 2;
  const int epb = pairs <= kScatterBlock ? kScatterBlock / pairs : 1;
  const int sub = pairs <= kScatterBlock ? (int)threadIdx.x / pairs : 0;
  const int pair0 = pairs <= kScatterBlock ? (int)threadIdx.x - sub * pairs : (int)threadIdx.x;
  if (sub >= epb) return;
  const int64_t groups = (E + epb - 1) / epb;
  const int64_t step = (int64_t)U * gridDim.x;
  for (int pr = pair0; pr < pairs; pr += kScatterBlock) {
    int64_t l[U];  // the next trip's local offsets and map entries
    int2 id[U];
    auto load = [&](int64_t g) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t slot = (g + (int64_t)u * gridDim.x) * epb + sub;
        l[u] = g < groups && slot < E ? (int64_t)__ldg(order + slot) * Np + 2 * pr : -1;
        if (l[u] >= 0 && !chk(bs_pred_index(l[u] / Np, E), BS_CHK_SCATTER_ENTRY)) l[u] = -1;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        id[u] = l[u] >= 0 ? __ldcs(reinterpret_cast<const int2 *>(ids + l[u])) : make_int2(-1, -1);
        if (!chk(bs_pred_map_entry(id[u].x, NG), BS_CHK_SCATTER_ENTRY)) id[u].x = -1;
        if (!chk(bs_pred_map_entry(id[u].y, NG), BS_CHK_SCATTER_ENTRY)) id[u].y = -1;
      }
    };
    load(blockIdx.x);
    for (int64_t g = blockIdx.x; g < groups; g += step) {
      int64_t lc[U];
      int2 ic[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        lc[u] = l[u];
        ic[u] = id[u];
      }
      T a[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        a[u] = ic[u].x >= 0 ? qG[ic[u].x] : T(0);
        b[u] = ic[u].y >= 0 ? qG[ic[u].y] : T(0);
      }
      load(g + step);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (lc[u] < 0) continue;
        if (ic[u].x >= 0 && ic[u].y >= 0) {
          V2 v;
          v.x = a[u];
          v.y = b[u];
          __stcs(reinterpret_cast<V2 *>(qL + lc[u]), v);
        } else {  // masked entries stay untouched
          if (ic[u].x >= 0) __stcs(qL + lc[u], a[u]);
          if (ic[u].y >= 0) __stcs(qL + lc[u] + 1, b[u]);
        }
      }
    }
  }
}

template <typename T>
int launch_scatter(const bs_map *m, const T *qG, T *qL, cudaStream_t s) {
  const int Np = (m->N + 1) * (m->N + 1) * (m->N + 1);
  if (Np % 2 == 0 && ((uintptr_t)qL % 16) == 0 && ((uintptr_t)m->d_ids % 8) == 0) {
    constexpr int U = 2;
    auto kern = k_scatter2<T, U>;
    const int pairs = Np / 2;
    const int epb = pairs <= kScatterBlock ? kScatterBlock / pairs : 1;
    const int64_t groups = (m->E + epb - 1) / epb;
    int grid = stream_grid(groups, U, 1, blocks_per_sm(kern, kScatterBlock));
    if (grid < 1) return fail(BS_ERR_CUDA, "no device");
    kern<<<grid, kScatterBlock, 0, s>>>(m->E, m->NG, Np, m->d_elem_order, m->d_ids, qG, qL);
    BS_LAUNCH_CHECK();
    return BS_OK;
  }
  constexpr int U = 4;
  auto kern = k_scatter<T, U>;
  const int epb = Np <= kScatterBlock ? kScatterBlock / Np : 1;
  const int64_t groups = (m->E + epb - 1) / epb;
  int grid = stream_grid(groups, U, 1, blocks_per_sm(kern, kScatterBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  kern<<<grid, kScatterBlock, 0, s>>>(m->E, m->NG, Np, m->d_elem_order, m->d_ids, qG, qL);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

}  // namespace bs
