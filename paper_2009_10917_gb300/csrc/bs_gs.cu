// bs_gs.cu -- the scatter operator Z (eq. scatter_def) as a map object, and
// the C ABI entry points of BS6 (gather) and BS7 (scatter).
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "bs_gather.cuh"

namespace bs {

__global__ void k_valence(int64_t NG, const int32_t *__restrict__ row_starts,
                          int32_t *__restrict__ val) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = tid; g < NG; g += nth) val[g] = row_starts[g + 1] - row_starts[g];
}

static int check_map(const bs_map *m, const char *fn) {
  if (!m) return fail(BS_ERR_ARG, "%s: map is NULL", fn);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device)
    return fail(BS_ERR_ARG, "%s: map belongs to device %d, current is %d", fn, m->device, dev);
  return BS_OK;
}

static void free_map(bs_map *m) {
  if (!m) return;
  cudaFree(m->d_ids);
  cudaFree(m->d_row_starts);
  cudaFree(m->d_col_ids);
  cudaFree(m->d_tiles);
  cudaFree(m->d_elem_order);
  cudaFree(m->d_ids_f);
  cudaFree(m->d_sh_rows);
  cudaFree(m->d_sh_starts);
  cudaFree(m->d_sh_cols);
  cudaFree(m->d_sh_tiles);
  cudaFree(m->d_ag_info);
  cudaFree(m->d_ag_chunks);
  cudaFree(m->d_ag_blob);
  free(m);
}

template <typename T>
static int do_scatter(const bs_map *m, const T *qG, T *qL, void *stream, const char *fn) {
  if (int rc = check_map(m, fn)) return rc;
  if (m->NL == 0) return BS_OK;
  BS_ARG(qL != nullptr && (qG != nullptr || m->NG == 0), "%s: NULL vector", fn);
  return launch_scatter<T>(m, qG, qL, as_stream(stream));
}

template <typename T>
static int do_gather(const bs_map *m, const T *qL, T *qG, void *stream, const char *fn) {
  if (int rc = check_map(m, fn)) return rc;
  if (m->NG == 0) return BS_OK;
  BS_ARG(qG != nullptr && (qL != nullptr || m->NL == 0), "%s: NULL vector", fn);
  return launch_gather<T, false, EpNone>(m, qL, qG, nullptr, nullptr, nullptr, EpNone{},
                                         nullptr, as_stream(stream));
}

// Gather tiles over rows [0, nrows) of a CSR: at most kTileRows consecutive
// rows holding at most kTileNnz entries (a longer row gets a tile of its
// own); at least one (possibly empty) tile.  (first row, first entry) each.
static std::vector<int2> make_tiles(const std::vector<int32_t> &rs, int64_t nrows) {
  std::vector<int32_t> tiles;
  tiles.push_back(0);
  for (int64_t g = 0; g < nrows;) {
    int64_t r = g;
    while (r < nrows && r - g < kTileRows && rs[(size_t)r + 1] - rs[(size_t)g] <= kTileNnz) ++r;
    if (r == g) r = g + 1;
    tiles.push_back((int32_t)r);
    g = r;
  }
  if (tiles.size() == 1) tiles.push_back(0);
  std::vector<int2> out(tiles.size());
  for (size_t i = 0; i < tiles.size(); ++i) out[i] = make_int2(tiles[i], rs[(size_t)tiles[i]]);
  return out;
}

template <typename V>
static cudaError_t upload(V **d, const std::vector<V> &h, size_t pad = 0) {
  cudaError_t e = cudaMalloc(d, sizeof(V) * (h.size() + pad + (h.empty() && !pad ? 1 : 0)));
  if (e == cudaSuccess && !h.empty())
    e = cudaMemcpy(*d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace bs

using namespace bs;

extern "C" {

int bs_map_create(int32_t E, int32_t N, int64_t NG, const int32_t *h_l2g, bs_map **out) {
  BS_ARG(out != nullptr, "bs_map_create: out is NULL");
  *out = nullptr;
  BS_ARG(E >= 0 && N >= 1 && N <= 15, "bs_map_create: need E >= 0 and 1 <= N <= 15");
  BS_ARG(NG >= 0 && NG < INT32_MAX, "bs_map_create: NG out of int32 range");
  const int64_t Np = (int64_t)(N + 1) * (N + 1) * (N + 1);
  const int64_t NL = (int64_t)E * Np;
  BS_ARG(NL < INT32_MAX, "bs_map_create: N_L out of int32 range");
  BS_ARG(NL == 0 || h_l2g != nullptr, "bs_map_create: map is NULL");
  // counts per global node (and validation) -- the valence, diag(Z^T Z)
  std::vector<int32_t> rs((size_t)NG + 1, 0);
  int64_t nnz = 0;
  for (int64_t l = 0; l < NL; ++l) {
    const int32_t id = h_l2g[l];
    if (id < 0) continue;
    if (id >= NG) return fail(BS_ERR_ARG, "bs_map_create: l2g[%lld] = %d >= NG", (long long)l, id);
    ++rs[(size_t)id + 1];
    ++nnz;
  }
  for (int64_t g = 0; g < NG; ++g) rs[(size_t)g + 1] += rs[(size_t)g];
  // stable placement: ascending l within each row
  std::vector<int32_t> col((size_t)nnz);
  {
    std::vector<int32_t> fill(rs.begin(), rs.end() - 1);
    for (int64_t l = 0; l < NL; ++l) {
      const int32_t id = h_l2g[l];
      if (id >= 0) col[(size_t)fill[(size_t)id]++] = (int32_t)l;
    }
  }
  const std::vector<int2> tile_bounds = make_tiles(rs, NG);
  // the fused operator's encoding and the CSR of the rows with >= 2 copies
  std::vector<int32_t> ids_f((size_t)NL), sh_rows, sh_starts(1, 0), sh_cols;
  for (int64_t l = 0; l < NL; ++l) {
    const int32_t id = h_l2g[l];
    ids_f[(size_t)l] = id < 0 ? -1 : (rs[(size_t)id + 1] - rs[(size_t)id] == 1 ? -2 - id : id);
  }
  for (int64_t g = 0; g < NG; ++g) {
    const int32_t a = rs[(size_t)g], b = rs[(size_t)g + 1];
    if (b - a == 1) continue;  // valence 0 rows stay here: the gather writes their zero
    sh_rows.push_back((int32_t)g);
    sh_cols.insert(sh_cols.end(), col.begin() + a, col.begin() + b);
    sh_starts.push_back((int32_t)sh_cols.size());
  }
  const std::vector<int2> sh_tiles = make_tiles(sh_starts, (int64_t)sh_rows.size());
  // elements in the order of their smallest global index (ties keep storage
  // order); all-masked elements go last
  std::vector<int32_t> order((size_t)E);
  {
    std::vector<int32_t> key((size_t)E, INT32_MAX);
    for (int64_t l = 0; l < NL; ++l) {
      const int32_t id = h_l2g[l];
      int32_t &k = key[(size_t)(l / Np)];
      if (id >= 0 && id < k) k = id;
    }
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return key[(size_t)a] < key[(size_t)b]; });
  }
  bs_map *m = (bs_map *)calloc(1, sizeof(bs_map));
  if (!m) return fail(BS_ERR_ALLOC, "bs_map_create: host allocation");
  m->E = E;
  m->N = N;
  m->NL = NL;
  m->NG = NG;
  m->nnz = nnz;
  m->ntiles = (int64_t)tile_bounds.size() - 1;
  m->nsh = (int64_t)sh_rows.size();
  m->nnz_sh = (int64_t)sh_cols.size();
  m->nsh_tiles = (int64_t)sh_tiles.size() - 1;
  cudaError_t e = cudaGetDevice(&m->device);
  // +4 elements of padding so 128-bit loads of the map never leave the buffer
  if (e == cudaSuccess) e = cudaMalloc(&m->d_ids, sizeof(int32_t) * (NL + 4));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_row_starts, sizeof(int32_t) * (NG + 1));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_col_ids, sizeof(int32_t) * (nnz + 4));
  if (e == cudaSuccess && NL)
    e = cudaMemcpy(m->d_ids, h_l2g, sizeof(int32_t) * NL, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_row_starts, rs.data(), sizeof(int32_t) * (NG + 1),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nnz)
    e = cudaMemcpy(m->d_col_ids, col.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_tiles, sizeof(int2) * tile_bounds.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_tiles, tile_bounds.data(), sizeof(int2) * tile_bounds.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_elem_order, sizeof(int32_t) * (E > 0 ? E : 1));
  if (e == cudaSuccess && E)
    e = cudaMemcpy(m->d_elem_order, order.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = upload(&m->d_ids_f, ids_f, 4);
  if (e == cudaSuccess) e = upload(&m->d_sh_rows, sh_rows);
  if (e == cudaSuccess) e = upload(&m->d_sh_starts, sh_starts);
  if (e == cudaSuccess) e = upload(&m->d_sh_cols, sh_cols, 4);
  if (e == cudaSuccess) e = upload(&m->d_sh_tiles, sh_tiles);
  if (e == cudaSuccess && NG > 0) {  // the pipelined FP64 gather's tiles
    AgTiles T = build_async_tiles(rs, col, NL, NG);
    m->ag_ntiles = (int64_t)T.info.size() - 1;
    static_assert(sizeof(AgInfo) == sizeof(int4), "tile info is the kernel's int4");
    std::vector<int4> info(T.info.size());
    memcpy(info.data(), T.info.data(), sizeof(int4) * info.size());
    e = upload(&m->d_ag_info, info);
    if (e == cudaSuccess) e = upload(&m->d_ag_chunks, T.chunks, 4);
    std::vector<uint4> words(T.blob.size() / 8);
    if (!words.empty()) memcpy(words.data(), T.blob.data(), T.blob.size() * sizeof(uint16_t));
    if (e == cudaSuccess) e = upload(&m->d_ag_blob, words, 1);
  }
  if (e != cudaSuccess) {
    free_map(m);
    return fail(BS_ERR_CUDA, "bs_map_create: %s", cudaGetErrorString(e));
  }
  *out = m;
  return BS_OK;
}

int bs_map_destroy(bs_map *m) {
  free_map(m);
  return BS_OK;
}

int bs_map_info(const bs_map *m, int64_t *NL, int64_t *NG, int64_t *nnz) {
  BS_ARG(m != nullptr, "bs_map_info: map is NULL");
  if (NL) *NL = m->NL;
  if (NG) *NG = m->NG;
  if (nnz) *nnz = m->nnz;
  return BS_OK;
}

int bs_map_export(const bs_map *m, int32_t *h_row_starts, int32_t *h_col_ids) {
  if (int rc = check_map(m, "bs_map_export")) return rc;
  if (h_row_starts)
    BS_CUDA_TRY(cudaMemcpy(h_row_starts, m->d_row_starts, sizeof(int32_t) * (m->NG + 1),
                           cudaMemcpyDeviceToHost));
  if (h_col_ids && m->nnz)
    BS_CUDA_TRY(cudaMemcpy(h_col_ids, m->d_col_ids, sizeof(int32_t) * m->nnz,
                           cudaMemcpyDeviceToHost));
  return BS_OK;
}

int bs_map_valence(const bs_map *m, int32_t *d_val, void *stream) {
  if (int rc = check_map(m, "bs_map_valence")) return rc;
  if (m->NG == 0) return BS_OK;
  BS_ARG(d_val != nullptr, "bs_map_valence: NULL output");
  const int grid = stream_grid(m->NG, 1, kStreamBlock, 8);
  k_valence<<<grid, kStreamBlock, 0, as_stream(stream)>>>(m->NG, m->d_row_starts, d_val);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

int bs_scatter(const bs_map *m, const double *qG, double *qL, void *stream) {
  return do_scatter<double>(m, qG, qL, stream, "bs_scatter");
}
int bs_scatter_f32(const bs_map *m, const float *qG, float *qL, void *stream) {
  return do_scatter<float>(m, qG, qL, stream, "bs_scatter_f32");
}
int bs_gather(const bs_map *m, const double *qL, double *qG, void *stream) {
  return do_gather<double>(m, qL, qG, stream, "bs_gather");
}
int bs_gather_f32(const bs_map *m, const float *qL, float *qG, void *stream) {
  return do_gather<float>(m, qL, qG, stream, "bs_gather_f32");
}

}  // extern "C"
