// bs_mlp.cuh -- the learned element preconditioner's network: y = W2 relu(W1 x)
// (no biases) with BF16 weights and activations on the tensor cores, FP32
// accumulation, FP32 master weights trained by Adam.
//
// Every product is one "TN" GEMM, C[M x N] = A[M x K] B[N x K]^T with A and B
// row-major bfloat16 (K contiguous, K a multiple of 32): 128 x 128 block
// tiles, 32-wide K steps double-buffered in shared memory by 16-byte
// cp.async, fragments loaded with ldmatrix, mma.sync m16n8k16 bf16 -> fp32.
// Epilogues are fused: hidden activation (ReLU or identity) to bf16, plain
// fp32, masked (relu') bf16, and the preconditioner's rms-scaled FP64
// element output.
//
// Precision modes.  BF16: weights and activations are single bf16 values.
// BF16x3: each is carried as hi + lo (hi = bf16(v), lo = bf16(v - hi)) and a
// product a b is formed as ahi bhi + ahi blo + alo bhi on the same BF16
// tensor cores, by one GEMM over a tripled K: rows of the activation operand
// are [hi | hi | lo] and rows of the weight operand [hi | lo | hi].  The
// relative error per product drops from about 2^-8 to about 2^-16, which an
// accurate local inverse of a high-order element (condition number in the
// hundreds) needs; the backward pass always uses the hi parts.
#pragma once

#include <cuda_bf16.h>

#include "bs_op.cuh"

struct bs_mlp {
  int device;
  int D, Dp, H;                     // Dp = D rounded up to a multiple of 32
  int split;                        // 1: BF16x3 mode (K tripled), 0: BF16
  float *W1, *W2;                   // FP32 master weights, W1 [H x Dp], W2 [Dp x H]
  float *m1, *v1, *m2, *v2;         // Adam moments
  // bf16 operands: W1b [H x K1], W2b [Dp x K2] (K1 = Dp, K2 = H, tripled in
  // BF16x3 mode as [hi | lo | hi]) and W2tb = hi(W2)^T [H x Dp]
  __nv_bfloat16 *W1b, *W2b, *W2tb;
  int step;                         // Adam steps taken
  // training scratch for batches of up to Bcap rows: Xb [B x K1], Hb [B x K2]
  // (activation operands, [hi | hi | lo] rows in BF16x3 mode), the rest bf16
  int64_t Bcap;
  __nv_bfloat16 *Xb, *Xtb, *Hb, *Htb, *dYb, *dYtb, *dZtb;
  float *Y, *g1, *g2;
  double *lossp;                    // per-block loss partials + counter
  unsigned int *cnt;
  // the odd part collapsed to one matrix L = W2 W1 / 2 [Dp x Dp] (FP32, from
  // the masters in FP64 sums) and its weight operand Lb [Dp x K1]; formed by
  // mlp_odd_matrix, valid while odd_step == step
  float *L;
  __nv_bfloat16 *Lb;
  int odd_step;
  // element-interior outputs: when D = (N+1)^3 with N >= 2, the nI = (N-1)^3
  // local indices lidx of the interior nodes and Wint [nI x max(K1, K2)], the
  // weight rows that produce them (rows of Lb for the odd part, of W2b for
  // the full network), formed by mlp_interior_operand
  int nI;
  int32_t *lidx;
  __nv_bfloat16 *Wint;
  int int_step, int_odd;
};

namespace bs {

enum GemmEpi {
  EPI_F32 = 0,       // out_f32[m ldc + n] = acc
  EPI_HIDDEN = 1,    // a = relu ? max(acc, 0) : acc; out_b16[m ldc + n] = bf16(a), and
                     // with split > 0 also hi at +split and lo = bf16(a - hi) at +2 split
  EPI_MASK_BF16 = 2, // out_b16[m ldc + n] = mask[m ldmask + n] > 0 ? bf16(acc) : 0
  EPI_SCALE_F64 = 3, // n < nvalid: out_f64[m ldc + n] = acc * scale[m]
  EPI_SCATTER_F64 = 4 // n < nvalid, gid = ids[order[m] np + lidx[n]] >= 0:
                      // out_f64[gid] = acc * scale[m]
};

// hi/lo bf16 split of a float (lo = 0 unless split)
__device__ __forceinline__ void bf16_split(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

struct GemmArgs {
  const __nv_bfloat16 *A, *B;  // A [M x K], B [N x K], row-major
  int64_t M;
  int N, K, lda, ldb, ldc, nvalid;
  float *out_f32;
  __nv_bfloat16 *out_b16;
  double *out_f64;
  const __nv_bfloat16 *mask;
  int ldmask, relu, split;
  const double *scale;  // EPI_SCALE_F64 / EPI_SCATTER_F64: per-row factor
  const int32_t *ids, *order, *lidx;  // EPI_SCATTER_F64: map, row -> element, local indices
  int np;
  int64_t ng;         // EPI_SCATTER_F64: length of out_f64 (checked build)
  const CgState *st;  // optional: skip the launch when a solve has stopped
  int *err;           // optional: set to 2 if a tensor-core wait gives up
};

// Epilogue of one accumulator value v at (m, n) (idrow: the map row of
// element order[m], EPI_SCATTER_F64 only).
template <int EPI>
__device__ __forceinline__ void gemm_store(const GemmArgs &g, int64_t m, int n, float v,
                                           const int32_t *idrow) {
  const int64_t o = m * g.ldc + n;
  if (EPI == EPI_F32) {
    g.out_f32[o] = v;
  } else if (EPI == EPI_HIDDEN) {
    __nv_bfloat16 hi, lo;
    bf16_split(g.relu ? (v > 0.f ? v : 0.f) : v, hi, lo);
    g.out_b16[o] = hi;
    if (g.split) {
      g.out_b16[o + g.split] = hi;
      g.out_b16[o + 2 * g.split] = lo;
    }
  } else if (EPI == EPI_MASK_BF16) {
    g.out_b16[o] = __bfloat162float(g.mask[m * g.ldmask + n]) > 0.f ? __float2bfloat16_rn(v)
                                                                    : __float2bfloat16_rn(0.f);
  } else if (EPI == EPI_SCALE_F64) {
    if (n < g.nvalid) g.out_f64[o] = (double)v * g.scale[m];
  } else {
    if (n < g.nvalid) {
      if (BS_CHECK && !idrow) return;  // element index failed its check
      const int lx = g.lidx[n];
      if (!chk(bs_pred_index(lx, g.np), BS_CHK_PREC_ENTRY)) return;
      int32_t gid = idrow[lx];
      if (!chk(bs_pred_map_entry(gid, g.ng), BS_CHK_PREC_ENTRY)) gid = -1;
      if (gid >= 0) g.out_f64[gid] = (double)v * g.scale[m];
    }
  }
}

// The tcgen05 path (bs_tc.cu): whether a GEMM can take it, and its launch.
bool gemm_tc_supported(int epi, const GemmArgs &a);
int launch_gemm_tc(int epi, const GemmArgs &a, int *err, cudaStream_t s);

int launch_gemm(int epi, const GemmArgs &a, cudaStream_t s);
// Hidden layer then output layer on the activation operand m->Xb (B rows,
// packed for the mlp's mode): Hb = act(Xb W1^T), then out = Hb W2^T through
// the given epilogue arguments (out_f32 or out_f64 + scale + nvalid, ldc).
int mlp_forward_packed(bs_mlp *m, int64_t B, int relu, GemmArgs out, int out_epi,
                       cudaStream_t s);


// Training/inference scratch for batches (or element counts) up to B rows.
int mlp_ensure(bs_mlp *m, int64_t B);
// L = W2 W1 / 2 and its operand Lb, if the weights changed since last formed.
int mlp_odd_matrix(bs_mlp *m, cudaStream_t s);
// Wint for the odd part (odd) or the full network's output layer, if stale.
int mlp_interior_operand(bs_mlp *m, int odd, cudaStream_t s);

}  // namespace bs
