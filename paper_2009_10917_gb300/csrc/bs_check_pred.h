/* Index predicates of the checked build (compiled with -DBS_CHECK=1).
 *
 * Every index a kernel takes from memory (a map entry, a CSR row bound or
 * column, a tile bound, a chunk id or an offset into a staged tile) is tested
 * by one of these before it is used.  They are plain C so that the host
 * tests compile and exercise the same definitions; under nvcc they are
 * host and device functions.  Each returns 1 when the index is valid.
 */
#ifndef BS_CHECK_PRED_H
#define BS_CHECK_PRED_H

#include <stdint.h>

#if defined(__CUDACC__)
#define BS_PRED __host__ __device__ __forceinline__
#else
#define BS_PRED static inline
#endif

/* 0 <= i < n: a position inside an array of n values. */
BS_PRED int bs_pred_index(int64_t i, int64_t n) { return i >= 0 && i < n; }

/* A local-to-global map entry (Sec. 5, scatterIds): a global index below
 * n_global, or any negative value (a masked local node). */
BS_PRED int bs_pred_map_entry(int64_t id, int64_t n_global) { return id < n_global; }

/* The fused operator's re-encoded map entry: id >= 0 is a node with a single
 * copy (written in place), -1 a masked node, -2 - g a shared node g; every
 * node index below n_global. */
BS_PRED int bs_pred_fused_entry(int64_t code, int64_t n_global) {
  return code < n_global && code > -2 - n_global;
}

/* A CSR row [b0, b1) inside the nnz column entries: 0 <= b0 <= b1 <= nnz. */
BS_PRED int bs_pred_row(int64_t b0, int64_t b1, int64_t nnz) {
  return b0 >= 0 && b0 <= b1 && b1 <= nnz;
}

/* A tile of rows [r0, r1) and entries [k0, k1) of a CSR with n_rows rows and
 * nnz entries, holding at most max_entries entries unless it is a single
 * row (a row longer than a tile is read straight from memory). */
BS_PRED int bs_pred_tile(int64_t r0, int64_t r1, int64_t k0, int64_t k1, int64_t n_rows,
                         int64_t nnz, int64_t max_entries) {
  return r0 >= 0 && r0 <= r1 && r1 <= n_rows && k0 >= 0 && k0 <= k1 && k1 <= nnz &&
         (k1 - k0 <= max_entries || r1 - r0 == 1);
}

/* An offset into a staged tile of n_staged values. */
BS_PRED int bs_pred_staged(int64_t off, int64_t n_staged) { return off >= 0 && off < n_staged; }

#undef BS_PRED

/* Codes recorded by a failed check (the first failure per translation unit
 * is kept; bs_check_device reports it). */
enum {
  BS_CHK_SCATTER_ENTRY = 1,  /* BS7: map entry >= N_G                          */
  BS_CHK_GATHER_TILE = 2,    /* BS6: tile bounds outside the CSR                */
  BS_CHK_GATHER_ROW = 3,     /* BS6: row bounds outside [0, nnz] or decreasing  */
  BS_CHK_GATHER_COL = 4,     /* BS6: column >= N_L                              */
  BS_CHK_GATHER_CHUNK = 5,   /* pipelined BS6: chunk id outside q_L             */
  BS_CHK_GATHER_STAGED = 6,  /* pipelined BS6: offset outside the staged tile   */
  BS_CHK_OP_ENTRY = 7,       /* element operator: map entry >= N_G              */
  BS_CHK_PREC_ENTRY = 8,     /* preconditioners, network epilogue: map entry    */
  BS_CHK_ROWS = 9,           /* multi-rank rows: row or column out of range     */
  BS_CHK_BATCH = 10          /* batched solver: item or element out of range    */
};

#endif
