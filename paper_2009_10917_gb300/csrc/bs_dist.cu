// bs_dist.cu -- the per-rank pieces of a gather (BS6) whose elements are
// split over several ranks (Sec. 3 sets the multi-rank gather aside as the
// non-trivial parallel implementation; this is this library's form of it).
//
// Each rank holds a contiguous range of the element storage order and a map
// of those elements onto the global nodes it touches.  A global node with
// copies on several ranks is summed as a chain in rank order: the first
// holder sums its copies from +0 (the ordinary gather), every later holder
// continues the serial sum from the partial it receives, and the last holder
// has the value the single-domain gather computes -- bit for bit, because the
// single-domain sum runs over ascending local index and every local index of
// a lower rank precedes every local index of a higher one.  The exchange
// itself is host-driven (paper_2009_10917_gb300/dist.py); this file provides
// the device steps: the continued sum of a set of rows, and packing and
// unpacking the values of a set of rows into contiguous message buffers.
#include <cstdlib>
#include <vector>

#include "bs_gather.cuh"

struct bs_rows {
  int device;
  const bs_map *map;
  int64_t n;
  int32_t *d_rows;  // [n] distinct rows of the map's Z^T, in message order
};

namespace bs {

constexpr int kRowsBlock = 256;

// qG[rows[i]] = (start ? start[i] : +0) + the row's copies in ascending
// local order, one serial sum per thread.  With start == NULL the first term
// enters as +0.0 + q (a -0.0 copy becomes +0.0), as in the gather.  gb
// bounds the indices in the checked build.
__global__ void __launch_bounds__(kRowsBlock)
    k_gather_rows(int64_t n, GBounds gb, const int32_t *__restrict__ rows,
                  const int32_t *__restrict__ row_starts, const int32_t *__restrict__ col_ids,
                  const double *__restrict__ qL, const double *__restrict__ start,
                  double *__restrict__ qG) {
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nth) {
    const int32_t g = rows[i];
    if (!chk(bs_pred_index(g, gb.ng), BS_CHK_ROWS)) continue;
    int32_t a = row_starts[g], b = row_starts[g + 1];
    if (!chk(bs_pred_row(a, b, gb.nnz), BS_CHK_ROWS)) a = b = 0;
    double s;
    int32_t k = a;
    if (start) {
      s = start[i];
    } else {
      s = 0.0;
      if (a < b && chk(bs_pred_index(col_ids[a], gb.nl), BS_CHK_ROWS))
        s = plus_zero(qL[col_ids[a]]);
      k = a + 1;
    }
    for (; k < b; ++k) {
      const int32_t c = col_ids[k];
      if (chk(bs_pred_index(c, gb.nl), BS_CHK_ROWS)) s = s + qL[c];
    }
    qG[g] = s;
  }
}

// buf[i] = qG[rows[i]] (PACK) or qG[rows[i]] = buf[i]; ng: length of qG.
template <bool PACK>
__global__ void __launch_bounds__(kRowsBlock)
    k_rows_move(int64_t n, int64_t ng, const int32_t *__restrict__ rows,
                const double *__restrict__ src, double *__restrict__ dst) {
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nth) {
    if (!chk(bs_pred_index(rows[i], ng), BS_CHK_ROWS)) continue;
    if (PACK)
      dst[i] = src[rows[i]];
    else
      dst[rows[i]] = src[i];
  }
}

static int check_rows(const bs_rows *rs, const char *fn) {
  if (!rs) return fail(BS_ERR_ARG, "%s: row set is NULL", fn);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != rs->device)
    return fail(BS_ERR_ARG, "%s: row set belongs to device %d, current is %d", fn, rs->device,
                dev);
  return BS_OK;
}

static int rows_grid(int64_t n) { return stream_grid(n, 1, kRowsBlock, 4); }

}  // namespace bs

using namespace bs;

extern "C" {

int bs_rows_create(const bs_map *m, int64_t nrows, const int32_t *h_rows, bs_rows **out) {
  BS_ARG(out != nullptr, "bs_rows_create: out is NULL");
  *out = nullptr;
  BS_ARG(m != nullptr, "bs_rows_create: map is NULL");
  BS_ARG(nrows >= 0 && nrows <= m->NG, "bs_rows_create: nrows %lld not in [0, NG]",
         (long long)nrows);
  BS_ARG(nrows == 0 || h_rows != nullptr, "bs_rows_create: rows is NULL");
  int dev = -1;
  BS_CUDA_TRY(cudaGetDevice(&dev));
  BS_ARG(dev == m->device, "bs_rows_create: map belongs to device %d, current is %d", m->device,
         dev);
  std::vector<unsigned char> seen((size_t)m->NG, 0);
  for (int64_t i = 0; i < nrows; ++i) {
    const int32_t g = h_rows[i];
    if (g < 0 || g >= m->NG)
      return fail(BS_ERR_ARG, "bs_rows_create: rows[%lld] = %d outside [0, %lld)", (long long)i,
                  g, (long long)m->NG);
    if (seen[(size_t)g]++)
      return fail(BS_ERR_ARG, "bs_rows_create: row %d listed twice", g);
  }
  bs_rows *rs = (bs_rows *)calloc(1, sizeof(bs_rows));
  if (!rs) return fail(BS_ERR_ALLOC, "bs_rows_create: host allocation");
  rs->device = dev;
  rs->map = m;
  rs->n = nrows;
  cudaError_t e = cudaMalloc(&rs->d_rows, sizeof(int32_t) * (size_t)(nrows > 0 ? nrows : 1));
  if (e == cudaSuccess && nrows > 0)
    e = cudaMemcpy(rs->d_rows, h_rows, sizeof(int32_t) * (size_t)nrows, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(rs->d_rows);
    free(rs);
    return fail(BS_ERR_CUDA, "bs_rows_create: %s", cudaGetErrorString(e));
  }
  *out = rs;
  return BS_OK;
}

int bs_rows_destroy(bs_rows *rs) {
  if (!rs) return BS_OK;
  cudaError_t e = cudaFree(rs->d_rows);
  free(rs);
  if (e != cudaSuccess) return fail(BS_ERR_CUDA, "bs_rows_destroy: %s", cudaGetErrorString(e));
  return BS_OK;
}

int bs_gather_rows(const bs_rows *rs, const double *qL, const double *start, double *qG,
                   void *stream) {
  if (int rc = check_rows(rs, "bs_gather_rows")) return rc;
  if (rs->n == 0) return BS_OK;
  BS_ARG(qG != nullptr && (qL != nullptr || rs->map->NL == 0), "bs_gather_rows: NULL vector");
  const int grid = rows_grid(rs->n);
  if (grid < 1) return fail(BS_ERR_CUDA, "bs_gather_rows: no device");
  k_gather_rows<<<grid, kRowsBlock, 0, as_stream(stream)>>>(
      rs->n, GBounds{rs->map->NG, rs->map->nnz, rs->map->NL, rs->map->NG}, rs->d_rows,
      rs->map->d_row_starts, rs->map->d_col_ids, qL, start, qG);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

int bs_rows_pack(const bs_rows *rs, const double *qG, double *buf, void *stream) {
  if (int rc = check_rows(rs, "bs_rows_pack")) return rc;
  if (rs->n == 0) return BS_OK;
  BS_ARG(qG != nullptr && buf != nullptr, "bs_rows_pack: NULL vector");
  const int grid = rows_grid(rs->n);
  if (grid < 1) return fail(BS_ERR_CUDA, "bs_rows_pack: no device");
  k_rows_move<true><<<grid, kRowsBlock, 0, as_stream(stream)>>>(rs->n, rs->map->NG, rs->d_rows,
                                                                qG, buf);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

int bs_rows_unpack(const bs_rows *rs, const double *buf, double *qG, void *stream) {
  if (int rc = check_rows(rs, "bs_rows_unpack")) return rc;
  if (rs->n == 0) return BS_OK;
  BS_ARG(qG != nullptr && buf != nullptr, "bs_rows_unpack: NULL vector");
  const int grid = rows_grid(rs->n);
  if (grid < 1) return fail(BS_ERR_CUDA, "bs_rows_unpack: no device");
  k_rows_move<false><<<grid, kRowsBlock, 0, as_stream(stream)>>>(rs->n, rs->map->NG, rs->d_rows,
                                                                 buf, qG);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

}  // extern "C"
