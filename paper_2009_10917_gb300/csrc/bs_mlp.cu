// bs_mlp.cu -- BF16 tensor-core GEMM and the MLP's forward pass, MSE loss and
// gradients, and Adam (see bs_mlp.cuh).  Training runs entirely in these
// kernels: forward (2 GEMMs), loss, backward (3 GEMMs), Adam, bf16 refresh.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "bs_mlp.cuh"

namespace bs {

constexpr int GBM = 128, GBK = 32, GPAD = 8;
constexpr int GTHREADS = 256;

__device__ __forceinline__ void cp_async16_zfill(void *smem, const void *gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t *r, const void *smem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float *c, const uint32_t *a, const uint32_t *b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C = A B^T on one 128 x BN tile per block (BN = 128 or 64); 8 warps as
// 2 (M) x 4 (N) warps of 64 x 32 for BN = 128, 4 x 2 warps of 32 x 32 for
// BN = 64 (outputs narrower than 64, as the 64 element-interior outputs of a
// degree-5 element, would waste half of a 128-wide tile).
template <int EPI, int BN>
__global__ void __launch_bounds__(GTHREADS) k_gemm_tn(GemmArgs g) {
  constexpr int WM = BN == 128 ? 2 : 4, WN = 8 / WM;
  constexpr int TM = GBM / WM, TN = BN / WN, MT = TM / 16, NT = TN / 8;
  static_assert(NT % 2 == 0 && MT >= 1, "warp tile");
  __shared__ __align__(16) __nv_bfloat16 sA[2][GBM][GBK + GPAD];
  __shared__ __align__(16) __nv_bfloat16 sB[2][BN][GBK + GPAD];
  if (cg_halted(g.st)) return;
  const int64_t m0 = (int64_t)blockIdx.y * GBM;
  const int n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp / WN, wn = warp % WN;
  float acc[MT][NT][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
  auto load = [&](int stage, int k0) {
#pragma unroll
    for (int c = tid; c < GBM * 4; c += GTHREADS) {
      const int row = c >> 2, col = (c & 3) * 8;
      const int64_t gm = m0 + row;
      const bool okA = gm < g.M;
      cp_async16_zfill(&sA[stage][row][col], g.A + (okA ? gm : 0) * g.lda + k0 + col, okA ? 16 : 0);
    }
#pragma unroll
    for (int c = tid; c < BN * 4; c += GTHREADS) {
      const int row = c >> 2, col = (c & 3) * 8;
      const int gn = n0 + row;
      const bool okB = gn < g.N;
      cp_async16_zfill(&sB[stage][row][col], g.B + (int64_t)(okB ? gn : 0) * g.ldb + k0 + col,
                       okB ? 16 : 0);
    }
  };
  const int nk = g.K / GBK;
  load(0, 0);
  cp_commit();
  for (int kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) load((kt + 1) & 1, (kt + 1) * GBK);
    cp_commit();
    cp_wait1();
    __syncthreads();
    const int st = kt & 1;
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t af[MT][4], bfr[NT][2];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
        ldmatrix_x4(af[mt], &sA[st][wm * TM + mt * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
      for (int np = 0; np < NT / 2; ++np) {
        uint32_t r[4];
        ldmatrix_x4(r, &sB[st][wn * TN + np * 16 + (lane & 7) + ((lane >> 4) << 3)]
                         [kk + ((lane >> 3) & 1) * 8]);
        bfr[2 * np][0] = r[0];
        bfr[2 * np][1] = r[1];
        bfr[2 * np + 1][0] = r[2];
        bfr[2 * np + 1][1] = r[3];
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt]);
    }
    __syncthreads();
  }
  const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t m = m0 + wm * TM + mt * 16 + gq + 8 * h;
      if (m >= g.M) continue;
      const int32_t *idrow = nullptr;
      if (EPI == EPI_SCATTER_F64) {
        const int64_t em = g.order ? g.order[m] : m;
        idrow = chk(bs_pred_index(em, g.M), BS_CHK_PREC_ENTRY) ? g.ids + em * g.np : nullptr;
      }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int n = n0 + wn * TN + nt * 8 + 2 * tq;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (n + e >= g.N) continue;
          gemm_store<EPI>(g, m, n + e, acc[mt][nt][2 * h + e], idrow);
        }
      }
    }
}

template <int EPI>
static void launch_epi(const GemmArgs &a, int64_t gy, cudaStream_t s) {
  if (a.N <= 64) {
    k_gemm_tn<EPI, 64><<<dim3((unsigned)((a.N + 63) / 64), (unsigned)gy), GTHREADS, 0, s>>>(a);
  } else {
    k_gemm_tn<EPI, 128><<<dim3((unsigned)((a.N + 127) / 128), (unsigned)gy), GTHREADS, 0, s>>>(a);
  }
}

int launch_gemm(int epi, const GemmArgs &a, cudaStream_t s) {
  if (a.K % GBK) return fail(BS_ERR_ARG, "gemm: K = %d is not a multiple of %d", a.K, GBK);
  if (a.M <= 0 || a.N <= 0) return BS_OK;
  if (gemm_tc_supported(epi, a)) return launch_gemm_tc(epi, a, a.err, s);
  const int64_t gy = (a.M + GBM - 1) / GBM;
  if (gy > 65535) return fail(BS_ERR_ARG, "gemm: M too large");
  switch (epi) {
    case EPI_F32: launch_epi<EPI_F32>(a, gy, s); break;
    case EPI_HIDDEN: launch_epi<EPI_HIDDEN>(a, gy, s); break;
    case EPI_MASK_BF16: launch_epi<EPI_MASK_BF16>(a, gy, s); break;
    case EPI_SCALE_F64: launch_epi<EPI_SCALE_F64>(a, gy, s); break;
    case EPI_SCATTER_F64: launch_epi<EPI_SCATTER_F64>(a, gy, s); break;
    default: return fail(BS_ERR_ARG, "gemm: unknown epilogue");
  }
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// ------------------------------------------------------------ small kernels

// Activation operand rows from in [R x C] float, padded to Cp columns with
// zeros: [hi] (row length Cp) or, with split, [hi | hi | lo] (3 Cp).
__global__ void k_pack_bf16(int64_t R, int C, int Cp, int split, const float *__restrict__ in,
                            __nv_bfloat16 *__restrict__ out) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t ld = split ? 3 * Cp : Cp;
  for (int64_t i = tid; i < R * Cp; i += nth) {
    const int64_t r = i / Cp;
    const int c = (int)(i - r * Cp);
    __nv_bfloat16 hi, lo;
    bf16_split(c < C ? in[r * C + c] : 0.f, hi, lo);
    out[r * ld + c] = hi;
    if (split) {
      out[r * ld + Cp + c] = hi;
      out[r * ld + 2 * Cp + c] = lo;
    }
  }
}

// out[c * R + r] = in[r * ldi + c] for r < R, c < C (bf16 transpose by tiles).
__global__ void k_transpose_bf16(int R, int C, int ldi, const __nv_bfloat16 *__restrict__ in,
                                 __nv_bfloat16 *__restrict__ out) {
  __shared__ __nv_bfloat16 t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < R && c < C) t[k][threadIdx.x] = in[(int64_t)r * ldi + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (r < R && c < C) out[(int64_t)c * R + r] = t[threadIdx.x][k];
  }
}

static int transpose(int R, int C, int ldi, const __nv_bfloat16 *in, __nv_bfloat16 *out,
                     cudaStream_t s) {
  dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
  k_transpose_bf16<<<grid, block, 0, s>>>(R, C, ldi, in, out);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// dY = 2 (Y - T) / (B D) as bf16 [B x Dp] (zero padding); loss = mean (Y - T)^2.
__global__ void __launch_bounds__(kReduceBlock)
    k_mse(int64_t B, int D, int Dp, const float *__restrict__ Y, const float *__restrict__ T,
          __nv_bfloat16 *__restrict__ dY, double *partials, unsigned int *counter,
          double *loss) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const float sc = (float)(2.0 / ((double)B * D));
  double acc = 0.0;
  for (int64_t i = tid; i < B * Dp; i += nth) {
    const int64_t r = i / Dp;
    const int c = (int)(i - r * Dp);
    float d = 0.f;
    if (c < D) {
      const float e = Y[i] - T[r * D + c];
      acc = fma((double)e, (double)e, acc);
      d = sc * e;
    }
    dY[i] = __float2bfloat16_rn(d);
  }
  const double part = block_sum<kReduceBlock>(acc);
  double total;
  if (grid_combine<kReduceBlock>(part, partials, counter, &total) && threadIdx.x == 0)
    *loss = total / ((double)B * D);
}

// Adam (Kingma & Ba 2015) on float weights; c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void k_adam(int64_t n, float *__restrict__ w, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += nth) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Weight operands from the FP32 masters: W1b rows [hi] or [hi | lo | hi]
// (row length K1 = Dp or 3 Dp), W2b likewise (K2 = H or 3 H), and
// W2tb = hi(W2)^T [H x Dp].
__global__ void k_refresh(int H, int Dp, int split, const float *__restrict__ W1,
                          const float *__restrict__ W2, __nv_bfloat16 *W1b, __nv_bfloat16 *W2b,
                          __nv_bfloat16 *W2tb) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t n = (int64_t)H * Dp;
  const int64_t K1 = split ? 3 * Dp : Dp, K2 = split ? 3 * H : H;
  for (int64_t i = tid; i < n; i += nth) {
    __nv_bfloat16 hi, lo;
    {  // W1 [H x Dp]
      const int64_t j = i / Dp, c = i - j * Dp;
      bf16_split(W1[i], hi, lo);
      W1b[j * K1 + c] = hi;
      if (split) {
        W1b[j * K1 + Dp + c] = lo;
        W1b[j * K1 + 2 * Dp + c] = hi;
      }
    }
    {  // W2 [Dp x H]
      const int64_t r = i / H, c = i - r * H;
      bf16_split(W2[i], hi, lo);
      W2b[r * K2 + c] = hi;
      if (split) {
        W2b[r * K2 + H + c] = lo;
        W2b[r * K2 + 2 * H + c] = hi;
      }
      W2tb[c * Dp + r] = hi;
    }
  }
}

// Y [B x D] (float) = scale * Y [B x Dp].
__global__ void k_unpad(int64_t B, int D, int Dp, float scale, const float *__restrict__ in,
                        float *__restrict__ out) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < B * D; i += nth) {
    const int64_t r = i / D;
    out[i] = scale * in[r * Dp + (i - r * D)];
  }
}

// gW [R x C] (float) from gP [R x ldp].
__global__ void k_unpad_cols(int R, int C, int ldp, const float *__restrict__ in,
                             float *__restrict__ out) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < (int64_t)R * C; i += nth) {
    const int64_t r = i / C;
    out[i] = in[r * ldp + (i - r * C)];
  }
}

// L [Dp x Dp] = W2 W1 / 2 (sums in FP64, rounded once to float; padded
// rows and columns are zero because the masters' padding is) and its weight
// operand Lb rows [hi] or [hi | lo | hi].
__global__ void k_odd_matrix(int H, int Dp, int split, const float *__restrict__ W1,
                             const float *__restrict__ W2, float *__restrict__ L,
                             __nv_bfloat16 *__restrict__ Lb) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t n = (int64_t)Dp * Dp, K1 = split ? 3 * Dp : Dp;
  for (int64_t i = tid; i < n; i += nth) {
    const int64_t r = i / Dp, c = i - r * Dp;
    double acc = 0.0;
    for (int j = 0; j < H; ++j) acc = fma((double)W2[r * H + j], (double)W1[(int64_t)j * Dp + c], acc);
    const float v = (float)(0.5 * acc);
    L[i] = v;
    __nv_bfloat16 hi, lo;
    bf16_split(v, hi, lo);
    Lb[r * K1 + c] = hi;
    if (split) {
      Lb[r * K1 + Dp + c] = lo;
      Lb[r * K1 + 2 * Dp + c] = hi;
    }
  }
}

// out rows n < nI: row lidx[n] of src (row length K, both operands; src
// has nsrc rows).
__global__ void k_rows(int nI, int K, int nsrc, const int32_t *__restrict__ lidx,
                       const __nv_bfloat16 *__restrict__ src, __nv_bfloat16 *__restrict__ out) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < (int64_t)nI * K; i += nth) {
    const int64_t n = i / K, k = i - n * K;
    if (!chk(bs_pred_index(lidx[n], nsrc), BS_CHK_PREC_ENTRY)) continue;
    out[i] = src[(int64_t)lidx[n] * K + k];
  }
}

int mlp_interior_operand(bs_mlp *m, int odd, cudaStream_t s) {
  if (m->nI <= 0) return fail(BS_ERR_ARG, "mlp: input size %d is not (N+1)^3 with N >= 2", m->D);
  if (m->int_step == m->step && m->int_odd == odd) return BS_OK;
  if (odd)
    if (int rc = mlp_odd_matrix(m, s)) return rc;
  const int K = odd ? (m->split ? 3 * m->Dp : m->Dp) : (m->split ? 3 * m->H : m->H);
  k_rows<<<stream_grid((int64_t)m->nI * K, 1, 256, 8), 256, 0, s>>>(
      m->nI, K, m->Dp, m->lidx, odd ? m->Lb : m->W2b, m->Wint);
  BS_LAUNCH_CHECK();
  m->int_step = m->step;
  m->int_odd = odd;
  return BS_OK;
}

int mlp_odd_matrix(bs_mlp *m, cudaStream_t s) {
  if (m->odd_step == m->step) return BS_OK;
  const int64_t n = (int64_t)m->Dp * m->Dp;
  k_odd_matrix<<<stream_grid(n, 1, 256, 8), 256, 0, s>>>(m->H, m->Dp, m->split, m->W1, m->W2,
                                                         m->L, m->Lb);
  BS_LAUNCH_CHECK();
  m->odd_step = m->step;
  return BS_OK;
}

static void free_scratch(bs_mlp *m) {
  cudaFree(m->Xb);
  cudaFree(m->Xtb);
  cudaFree(m->Hb);
  cudaFree(m->Htb);
  cudaFree(m->dYb);
  cudaFree(m->dYtb);
  cudaFree(m->dZtb);
  cudaFree(m->Y);
  m->Xb = m->Xtb = m->Hb = m->Htb = m->dYb = m->dYtb = m->dZtb = nullptr;
  m->Y = nullptr;
  m->Bcap = 0;
}

int mlp_ensure(bs_mlp *m, int64_t B) {
  if (B <= m->Bcap) return BS_OK;
  free_scratch(m);
  const int64_t Dp = m->Dp, H = m->H;
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  const int64_t k3 = m->split ? 3 : 1;
  A((void **)&m->Xb, 2 * B * Dp * k3);
  A((void **)&m->Xtb, 2 * B * Dp);
  A((void **)&m->Hb, 2 * B * H * k3);
  A((void **)&m->Htb, 2 * B * H);
  A((void **)&m->dYb, 2 * B * Dp);
  A((void **)&m->dYtb, 2 * B * Dp);
  A((void **)&m->dZtb, 2 * B * H);
  A((void **)&m->Y, 4 * B * Dp);
  if (e != cudaSuccess) {
    free_scratch(m);
    return fail(BS_ERR_ALLOC, "mlp scratch for %lld rows: %s", (long long)B, cudaGetErrorString(e));
  }
  m->Bcap = B;
  return BS_OK;
}

static int check_mlp(const bs_mlp *m, const char *fn) {
  if (!m) return fail(BS_ERR_ARG, "%s: mlp is NULL", fn);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device)
    return fail(BS_ERR_ARG, "%s: mlp belongs to device %d", fn, m->device);
  return BS_OK;
}

int mlp_forward_packed(bs_mlp *m, int64_t B, int relu, GemmArgs b, int out_epi, cudaStream_t s) {
  const int K1 = m->split ? 3 * m->Dp : m->Dp, K2 = m->split ? 3 * m->H : m->H;
  GemmArgs a{};
  a.A = m->Xb;
  a.B = m->W1b;
  a.M = B;
  a.N = m->H;
  a.K = K1;
  a.lda = K1;
  a.ldb = K1;
  a.ldc = K2;
  a.out_b16 = m->Hb;
  a.relu = relu;
  a.split = m->split ? m->H : 0;
  a.st = b.st;
  if (int rc = launch_gemm(EPI_HIDDEN, a, s)) return rc;
  b.A = m->Hb;
  b.B = m->W2b;
  b.M = B;
  b.N = m->Dp;
  b.K = K2;
  b.lda = K2;
  b.ldb = K2;
  return launch_gemm(out_epi, b, s);
}

// Forward of f on Xb: Y [B x Dp] (float).
static int forward_packed(bs_mlp *m, int64_t B, cudaStream_t s) {
  GemmArgs b{};
  b.ldc = m->Dp;
  b.out_f32 = m->Y;
  return mlp_forward_packed(m, B, 1, b, EPI_F32, s);
}

// Forward + MSE + backward into m->g1 (H x Dp), m->g2 (Dp x H) (float).
static int loss_grad(bs_mlp *m, int64_t B, const float *X, const float *T, double *d_loss,
                     cudaStream_t s) {
  const int Dp = m->Dp, H = m->H, D = m->D;
  const int K1 = m->split ? 3 * Dp : Dp, K2 = m->split ? 3 * H : H;
  const int grid = stream_grid(B * Dp, 1, 256, 8);
  k_pack_bf16<<<grid, 256, 0, s>>>(B, D, Dp, m->split, X, m->Xb);
  BS_LAUNCH_CHECK();
  if (int rc = forward_packed(m, B, s)) return rc;
  k_mse<<<stream_grid(B * Dp, 1, kReduceBlock, 4), kReduceBlock, 0, s>>>(
      B, D, Dp, m->Y, T, m->dYb, m->lossp, m->cnt, d_loss);
  BS_LAUNCH_CHECK();
  if (int rc = transpose((int)B, Dp, K1, m->Xb, m->Xtb, s)) return rc;   // hi(X)^T [Dp x B]
  if (int rc = transpose((int)B, H, K2, m->Hb, m->Htb, s)) return rc;    // hi(H)^T [H x B]
  if (int rc = transpose((int)B, Dp, Dp, m->dYb, m->dYtb, s)) return rc; // dY^T [Dp x B]
  // gW2 [Dp x H] = dY^T H
  GemmArgs g2{};
  g2.A = m->dYtb;
  g2.B = m->Htb;
  g2.M = Dp;
  g2.N = H;
  g2.K = (int)B;
  g2.lda = (int)B;
  g2.ldb = (int)B;
  g2.ldc = H;
  g2.out_f32 = m->g2;
  if (int rc = launch_gemm(EPI_F32, g2, s)) return rc;
  // dZ [B x H] = (dY W2) * relu'(hidden); W2 as B operand is W2^T [H x Dp]
  GemmArgs dz{};
  dz.A = m->dYb;
  dz.B = m->W2tb;
  dz.M = B;
  dz.N = H;
  dz.K = Dp;
  dz.lda = Dp;
  dz.ldb = Dp;
  dz.ldc = H;
  dz.out_b16 = m->Htb;  // reuse: H^T already consumed by gW2 above (same stream)
  dz.mask = m->Hb;
  dz.ldmask = K2;
  if (int rc = launch_gemm(EPI_MASK_BF16, dz, s)) return rc;
  if (int rc = transpose((int)B, H, H, m->Htb, m->dZtb, s)) return rc;   // dZ^T [H x B]
  // gW1 [H x Dp] = dZ^T X
  GemmArgs g1{};
  g1.A = m->dZtb;
  g1.B = m->Xtb;
  g1.M = H;
  g1.N = Dp;
  g1.K = (int)B;
  g1.lda = (int)B;
  g1.ldb = (int)B;
  g1.ldc = Dp;
  g1.out_f32 = m->g1;
  return launch_gemm(EPI_F32, g1, s);
}

static void free_mlp(bs_mlp *m) {
  if (!m) return;
  free_scratch(m);
  cudaFree(m->W1);
  cudaFree(m->L);
  cudaFree(m->lidx);
  cudaFree(m->lossp);
  free(m);
}

}  // namespace bs

using namespace bs;

extern "C" {

int bs_mlp_create(int32_t D, int32_t H, const float *h_W1, const float *h_W2, int32_t flags,
                  bs_mlp **out) {
  BS_ARG(out != nullptr, "bs_mlp_create: out is NULL");
  *out = nullptr;
  BS_ARG(D >= 1 && D <= 4096 && H >= 32 && H <= 4096 && H % 32 == 0,
         "bs_mlp_create: need 1 <= D <= 4096 and H a multiple of 32 in [32, 4096]");
  BS_ARG(h_W1 && h_W2, "bs_mlp_create: NULL weights");
  BS_ARG((flags & ~BS_MLP_BF16X3) == 0, "bs_mlp_create: unknown flags 0x%x", (unsigned)flags);
  bs_mlp *m = (bs_mlp *)calloc(1, sizeof(bs_mlp));
  if (!m) return fail(BS_ERR_ALLOC, "bs_mlp_create: host allocation");
  m->D = D;
  m->H = H;
  m->Dp = (D + 31) / 32 * 32;
  m->split = (flags & BS_MLP_BF16X3) ? 1 : 0;
  const size_t n = (size_t)H * m->Dp;
  // one allocation: W1, W2, m1, v1, m2, v2, g1, g2 (float) + bf16 operands
  // W1b (3n), W2b (3n), W2tb (n)
  cudaError_t e = cudaGetDevice(&m->device);
  char *base = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&base, n * (8 * sizeof(float) + 7 * 2) + 256);
  if (e == cudaSuccess) e = cudaMemset(base, 0, n * (8 * sizeof(float) + 7 * 2) + 256);
  {  // L (float Dp x Dp) then Lb (bf16 Dp x 3 Dp)
    const size_t nl = (size_t)m->Dp * m->Dp;
    if (e == cudaSuccess) e = cudaMalloc(&m->L, nl * (sizeof(float) + 3 * 2) + 256);
    m->Lb = m->L ? reinterpret_cast<__nv_bfloat16 *>(m->L + nl) : nullptr;
    m->odd_step = -1;
  }
  {  // interior local indices and their weight rows, when D = (N+1)^3, N >= 2
    int Nq = 1;
    while ((Nq + 1) * (Nq + 1) * (Nq + 1) <= D) ++Nq;
    m->nI = (Nq * Nq * Nq == D && Nq >= 3) ? (Nq - 2) * (Nq - 2) * (Nq - 2) : 0;
    m->int_step = -1;
    if (m->nI > 0 && e == cudaSuccess) {
      const int Kmax = 3 * (m->Dp > H ? m->Dp : H);
      int32_t *hl = (int32_t *)malloc(sizeof(int32_t) * m->nI);
      if (!hl) e = cudaErrorMemoryAllocation;
      int q = 0;
      for (int k = 1; hl && k < Nq - 1; ++k)
        for (int j = 1; j < Nq - 1; ++j)
          for (int i = 1; i < Nq - 1; ++i) hl[q++] = i + Nq * (j + Nq * k);
      if (e == cudaSuccess)
        e = cudaMalloc(&m->lidx, sizeof(int32_t) * m->nI + 256 + (size_t)m->nI * Kmax * 2);
      if (e == cudaSuccess) {
        m->Wint = reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<char *>(m->lidx) +
                                                    ((sizeof(int32_t) * m->nI + 255) / 256) * 256);
        e = cudaMemcpy(m->lidx, hl, sizeof(int32_t) * m->nI, cudaMemcpyHostToDevice);
      }
      free(hl);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->lossp, sizeof(double) * kMaxPartials + 256);
  if (e == cudaSuccess) e = cudaMemset(m->lossp, 0, sizeof(double) * kMaxPartials + 256);
  if (e != cudaSuccess) {
    if (base) cudaFree(base);
    free_mlp(m);
    return fail(BS_ERR_CUDA, "bs_mlp_create: %s", cudaGetErrorString(e));
  }
  float *f = reinterpret_cast<float *>(base);
  m->W1 = f;
  m->W2 = f + n;
  m->m1 = f + 2 * n;
  m->v1 = f + 3 * n;
  m->m2 = f + 4 * n;
  m->v2 = f + 5 * n;
  m->g1 = f + 6 * n;
  m->g2 = f + 7 * n;
  __nv_bfloat16 *bb = reinterpret_cast<__nv_bfloat16 *>(f + 8 * n);
  m->W1b = bb;
  m->W2b = bb + 3 * n;
  m->W2tb = bb + 6 * n;
  m->cnt = reinterpret_cast<unsigned int *>(m->lossp + kMaxPartials);
  // padded host copies -> device
  float *p1 = (float *)calloc(n, sizeof(float)), *p2 = (float *)calloc(n, sizeof(float));
  if (!p1 || !p2) {
    free(p1);
    free(p2);
    free_mlp(m);
    return fail(BS_ERR_ALLOC, "bs_mlp_create: host allocation");
  }
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < D; ++i) p1[(size_t)j * m->Dp + i] = h_W1[(size_t)j * D + i];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < H; ++j) p2[(size_t)i * H + j] = h_W2[(size_t)i * H + j];
  e = cudaMemcpy(m->W1, p1, n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->W2, p2, n * sizeof(float), cudaMemcpyHostToDevice);
  free(p1);
  free(p2);
  if (e != cudaSuccess) {
    free_mlp(m);
    return fail(BS_ERR_CUDA, "bs_mlp_create: %s", cudaGetErrorString(e));
  }
  k_refresh<<<stream_grid((int64_t)n, 1, 256, 8), 256>>>(H, m->Dp, m->split, m->W1, m->W2,
                                                          m->W1b, m->W2b, m->W2tb);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_mlp(m);
    return fail(BS_ERR_CUDA, "bs_mlp_create: %s", cudaGetErrorString(e));
  }
  *out = m;
  return BS_OK;
}

int bs_mlp_destroy(bs_mlp *m) {
  free_mlp(m);
  return BS_OK;
}

int bs_mlp_get_weights(const bs_mlp *m, float *h_W1, float *h_W2) {
  if (int rc = check_mlp(m, "bs_mlp_get_weights")) return rc;
  const size_t n = (size_t)m->H * m->Dp;
  float *p = (float *)malloc(2 * n * sizeof(float));
  if (!p) return fail(BS_ERR_ALLOC, "bs_mlp_get_weights: host allocation");
  cudaError_t e = cudaMemcpy(p, m->W1, 2 * n * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    free(p);
    return fail(BS_ERR_CUDA, "bs_mlp_get_weights: %s", cudaGetErrorString(e));
  }
  if (h_W1)
    for (int j = 0; j < m->H; ++j)
      for (int i = 0; i < m->D; ++i) h_W1[(size_t)j * m->D + i] = p[(size_t)j * m->Dp + i];
  if (h_W2)
    for (int i = 0; i < m->D; ++i)
      for (int j = 0; j < m->H; ++j) h_W2[(size_t)i * m->H + j] = p[n + (size_t)i * m->H + j];
  free(p);
  return BS_OK;
}

// Training-state image: a header, then W1, W2, m1, v1, m2, v2 as stored on
// the device (n = H * Dp floats each, padded layout).
struct MlpStateHeader {
  char magic[8];  // "BSMLPST1"
  int32_t D, Dp, H, split, step, reserved;
};
static const char kStateMagic[8] = {'B', 'S', 'M', 'L', 'P', 'S', 'T', '1'};

int64_t bs_mlp_state_bytes(const bs_mlp *m) {
  if (!m) return -1;
  return (int64_t)sizeof(MlpStateHeader) + 6 * (int64_t)m->H * m->Dp * (int64_t)sizeof(float);
}

int bs_mlp_save_state(const bs_mlp *m, void *h_buf, int64_t nbytes) {
  if (int rc = check_mlp(m, "bs_mlp_save_state")) return rc;
  BS_ARG(h_buf != nullptr, "bs_mlp_save_state: NULL buffer");
  BS_ARG(nbytes >= bs_mlp_state_bytes(m), "bs_mlp_save_state: buffer of %lld bytes, need %lld",
         (long long)nbytes, (long long)bs_mlp_state_bytes(m));
  MlpStateHeader h{};
  memcpy(h.magic, kStateMagic, 8);
  h.D = m->D;
  h.Dp = m->Dp;
  h.H = m->H;
  h.split = m->split;
  h.step = m->step;
  memcpy(h_buf, &h, sizeof(h));
  // W1, W2, m1, v1, m2, v2 are consecutive in the one allocation
  const size_t n = (size_t)m->H * m->Dp;
  BS_CUDA_TRY(cudaDeviceSynchronize());
  BS_CUDA_TRY(cudaMemcpy(static_cast<char *>(h_buf) + sizeof(h), m->W1, 6 * n * sizeof(float),
                         cudaMemcpyDeviceToHost));
  return BS_OK;
}

int bs_mlp_load_state(bs_mlp *m, const void *h_buf, int64_t nbytes) {
  if (int rc = check_mlp(m, "bs_mlp_load_state")) return rc;
  BS_ARG(h_buf != nullptr, "bs_mlp_load_state: NULL buffer");
  BS_ARG(nbytes >= (int64_t)sizeof(MlpStateHeader), "bs_mlp_load_state: buffer too short");
  MlpStateHeader h;
  memcpy(&h, h_buf, sizeof(h));
  BS_ARG(memcmp(h.magic, kStateMagic, 8) == 0, "bs_mlp_load_state: not a training-state image");
  BS_ARG(h.D == m->D && h.Dp == m->Dp && h.H == m->H && h.split == m->split,
         "bs_mlp_load_state: image is D %d H %d split %d, network is D %d H %d split %d", h.D,
         h.H, h.split, m->D, m->H, m->split);
  BS_ARG(h.step >= 0, "bs_mlp_load_state: negative step count");
  BS_ARG(nbytes >= bs_mlp_state_bytes(m), "bs_mlp_load_state: buffer of %lld bytes, need %lld",
         (long long)nbytes, (long long)bs_mlp_state_bytes(m));
  const size_t n = (size_t)m->H * m->Dp;
  BS_CUDA_TRY(cudaDeviceSynchronize());
  BS_CUDA_TRY(cudaMemcpy(m->W1, static_cast<const char *>(h_buf) + sizeof(h),
                         6 * n * sizeof(float), cudaMemcpyHostToDevice));
  m->step = h.step;
  m->odd_step = -1;  // derived operands are stale
  m->int_step = -1;
  k_refresh<<<stream_grid((int64_t)n, 1, 256, 8), 256>>>(m->H, m->Dp, m->split, m->W1, m->W2,
                                                          m->W1b, m->W2b, m->W2tb);
  BS_CUDA_TRY(cudaDeviceSynchronize());
  return BS_OK;
}

int bs_mlp_forward(bs_mlp *m, int64_t B, const float *d_X, float *d_Y, int32_t flags,
                   void *stream) {
  if (int rc = check_mlp(m, "bs_mlp_forward")) return rc;
  BS_ARG(B >= 0, "bs_mlp_forward: B < 0");
  if (B == 0) return BS_OK;
  BS_ARG(d_X && d_Y, "bs_mlp_forward: NULL vector");
  BS_ARG((flags & ~BS_MLP_ODD) == 0, "bs_mlp_forward: unknown flags 0x%x", (unsigned)flags);
  const int odd = (flags & BS_MLP_ODD) ? 1 : 0;
  if (int rc = mlp_ensure(m, B)) return rc;
  cudaStream_t s = as_stream(stream);
  k_pack_bf16<<<stream_grid(B * m->Dp, 1, 256, 8), 256, 0, s>>>(B, m->D, m->Dp, m->split, d_X,
                                                                 m->Xb);
  BS_LAUNCH_CHECK();
  GemmArgs b{};
  b.ldc = m->Dp;
  b.out_f32 = m->Y;
  // the odd part (f(x) - f(-x)) / 2 of a bias-free ReLU network is W2 W1 x / 2
  if (int rc = mlp_forward_packed(m, B, odd ? 0 : 1, b, EPI_F32, s)) return rc;
  k_unpad<<<stream_grid(B * m->D, 1, 256, 8), 256, 0, s>>>(B, m->D, m->Dp, odd ? 0.5f : 1.0f,
                                                           m->Y, d_Y);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

int bs_mlp_loss_grad(bs_mlp *m, int64_t B, const float *d_X, const float *d_T, double *d_loss,
                     float *d_gW1, float *d_gW2, void *stream) {
  if (int rc = check_mlp(m, "bs_mlp_loss_grad")) return rc;
  BS_ARG(B >= 32 && B % 32 == 0, "bs_mlp_loss_grad: batch must be a positive multiple of 32");
  BS_ARG(d_X && d_T && d_loss, "bs_mlp_loss_grad: NULL argument");
  if (int rc = mlp_ensure(m, B)) return rc;
  cudaStream_t s = as_stream(stream);
  if (int rc = loss_grad(m, B, d_X, d_T, d_loss, s)) return rc;
  if (d_gW1) {
    k_unpad_cols<<<stream_grid((int64_t)m->H * m->D, 1, 256, 8), 256, 0, s>>>(m->H, m->D, m->Dp,
                                                                              m->g1, d_gW1);
    BS_LAUNCH_CHECK();
  }
  if (d_gW2) {
    // g2 is [Dp x H]: the first D rows are the gradient
    BS_CUDA_TRY(cudaMemcpyAsync(d_gW2, m->g2, sizeof(float) * (size_t)m->D * m->H,
                                cudaMemcpyDeviceToDevice, s));
  }
  return BS_OK;
}

int bs_mlp_train_step(bs_mlp *m, int64_t B, const float *d_X, const float *d_T, float lr,
                      double *d_loss, void *stream) {
  if (int rc = check_mlp(m, "bs_mlp_train_step")) return rc;
  BS_ARG(B >= 32 && B % 32 == 0, "bs_mlp_train_step: batch must be a positive multiple of 32");
  BS_ARG(d_X && d_T && d_loss, "bs_mlp_train_step: NULL argument");
  BS_ARG(lr > 0.f && std::isfinite(lr), "bs_mlp_train_step: lr must be positive");
  if (int rc = mlp_ensure(m, B)) return rc;
  cudaStream_t s = as_stream(stream);
  if (int rc = loss_grad(m, B, d_X, d_T, d_loss, s)) return rc;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
  const int64_t n = (int64_t)m->H * m->Dp;
  const int grid = stream_grid(n, 1, 256, 8);
  k_adam<<<grid, 256, 0, s>>>(n, m->W1, m->g1, m->m1, m->v1, lr, b1, b2, eps, c1, c2);
  k_adam<<<grid, 256, 0, s>>>(n, m->W2, m->g2, m->m2, m->v2, lr, b1, b2, eps, c1, c2);
  k_refresh<<<grid, 256, 0, s>>>(m->H, m->Dp, m->split, m->W1, m->W2, m->W1b, m->W2b, m->W2tb);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

}  // extern "C"
