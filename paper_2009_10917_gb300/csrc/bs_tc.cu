// bs_tc.cu -- the network's GEMMs on the 5th-generation tensor cores
// (tcgen05): C[M x N] = A[M x K] B[N x K]^T, A and B row-major bf16 (K
// contiguous, K a multiple of 8), FP32 accumulation in tensor memory, and
// the epilogues of bs_mlp.cu.
//
// One CTA of 256 threads per 128-row tile and up to 256 output columns:
//  - K is consumed in 64-wide chunks through a 4-stage shared-memory ring
//    filled by 16-byte cp.async in the canonical K-major layout without
//    swizzle: 8-row x 16-byte core matrices, 128 bytes each, the eight core
//    matrices of a row group adjacent along K (leading byte offset 128) and
//    row groups 1024 bytes apart (stride byte offset 1024);
//  - one elected thread issues four tcgen05.mma (M = 128, N = the tile's
//    columns rounded up to 16, K = 16 each) per chunk and commits them to the
//    stage's mbarrier, which frees the stage for the chunk three ahead;
//  - the accumulator lives in tensor memory (one column per output column);
//    each warp reads its 32 rows (of 16-column chunks, shared by two warps)
//    back with tcgen05.ld (32x32b, 16 columns at a time) and applies the
//    epilogue.
// Every mbarrier wait is bounded: on expiry the kernel records an error
// (err, e.g. a solve's done flag, set to 2), still waits (bounded) for the
// MMAs it committed, frees its tensor memory and returns.
//
// Measured on GB300 against the mma.sync kernel of bs_mlp.cu (results are
// bitwise identical: both accumulate 16-wide K blocks in FP32 in the same
// order): the learned preconditioner's interior GEMM (M = E, N = 64,
// K = 672) takes 137 us against 97 us on the N = 5, 48^3 mesh, with 2, 3 or
// 4 stages alike.  Both kernels are bound by the latency of their loads and
// of the scattered epilogue, not by the tensor pipe (7% and 19% busy); this
// form has no TMA, no warp specialisation and no overlap of one tile's
// epilogue with the next tile's loads, which a faster tcgen05 path needs.
// So mma.sync is the default engine and this one is selected with
// bs_gemm_engine(1).
#include <mutex>

#include "bs_mlp.cuh"

namespace bs {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128, kTcK = 64, kTcMaxN = 256, kTcStages = 4;
constexpr int kTcStageA = kTcM * kTcK * 2;  // 16 KB
constexpr long long kTcWaitIters = 1ll << 22;

// Dynamic shared memory of a launch with npad columns: kTcStages stages of
// A (128 x 64) and B (npad x 64), then two mbarrier slots per stage and the
// TMEM address.
static inline int tc_smem_bytes(int npad) {
  return kTcStages * (kTcStageA + npad * kTcK * 2) + kTcStages * 8 + 16;
}

int g_gemm_engine = 0;  // 0: mma.sync (default, measured faster here); 1: tcgen05

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tc_cp_async16(void *smem, const void *gmem, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(bytes)
               : "memory");
}

// Shared-memory matrix descriptor (no swizzle): start address, leading and
// stride byte offsets (all >> 4), and the version field (1) at bits 46-47.
__device__ __forceinline__ uint64_t tc_desc(const void *smem, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = (smem_u32(smem) & 0x3FFFFu) >> 4;
  return a | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < kTcWaitIters; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// K is taken in 64-wide chunks (a last partial chunk is zero-filled past K).
// Layout of a stage: row r, 16-byte column chunk q (0..7) of a 64-wide K
// chunk at ((r / 8) * 8 + q) * 128 + (r % 8) * 16: core matrices 128 bytes
// apart along K (LBO), row groups 1024 bytes apart (SBO).
template <int EPI>
__global__ void __launch_bounds__(kTcThreads) k_gemm_tc(GemmArgs g, int *err) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  if (cg_halted(g.st)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * kTcM;
  const int n0 = blockIdx.y * kTcMaxN;
  const int nt = g.N - n0 < kTcMaxN ? g.N - n0 : kTcMaxN;  // valid columns of this tile
  const int npad = (nt + 15) & ~15;                        // MMA N
  const uint32_t ncols = npad <= 32 ? 32u : (npad <= 64 ? 64u : (npad <= 128 ? 128u : 256u));
  const int stage_bytes = kTcStageA + npad * kTcK * 2;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(tc_smem + kTcStages * stage_bytes);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(mbar + kTcStages);

  if (tid == 0) {
    for (int i = 0; i < kTcStages; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(s_tmem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *s_tmem;

  const int nk = (g.K + kTcK - 1) / kTcK;  // a last chunk past K is zero-filled
  auto load = [&](int chunk) {
    uint8_t *sA = tc_smem + (chunk % kTcStages) * stage_bytes, *sB = sA + kTcStageA;
    const int k0 = chunk * kTcK;
    // thread c -> row (c / 64) * 8 + c % 8, chunk (c / 8) % 8: eight
    // consecutive threads fill one 128-byte core matrix (no bank conflicts),
    // four of them cover 64 contiguous bytes of a row
    for (int c = tid; c < kTcM * 8; c += kTcThreads) {
      const int r = ((c >> 6) << 3) | (c & 7), q = (c >> 3) & 7;
      const int64_t gm = m0 + r;
      const bool ok = gm < g.M && k0 + q * 8 < g.K;
      tc_cp_async16(sA + ((r >> 3) * 8 + q) * 128 + (r & 7) * 16,
                    g.A + (ok ? gm * g.lda + k0 + q * 8 : 0), ok ? 16 : 0);
    }
    for (int c = tid; c < npad * 8; c += kTcThreads) {
      const int r = ((c >> 6) << 3) | (c & 7), q = (c >> 3) & 7;
      const bool ok = r < nt && k0 + q * 8 < g.K;
      tc_cp_async16(sB + ((r >> 3) * 8 + q) * 128 + (r & 7) * 16,
                    g.B + (ok ? (int64_t)(n0 + r) * g.ldb + k0 + q * 8 : 0), ok ? 16 : 0);
    }
  };
  // kind::f16, D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1),
  // both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(npad >> 3) << 17) |
                         ((uint32_t)(kTcM >> 4) << 24);
  int ok = 1, issued = 0;
  // prologue: chunks 0 .. kTcStages - 2 in flight, one cp.async group each
  for (int c = 0; c < kTcStages - 1; ++c) {
    if (c < nk) load(c);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int kt = 0; kt < nk; ++kt) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kTcStages - 2) : "memory");  // chunk kt landed
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    ok = __syncthreads_and(ok);
    if (!ok) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      uint8_t *sA = tc_smem + (kt % kTcStages) * stage_bytes, *sB = sA + kTcStageA;
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; ++kk) {
        const uint64_t ad = tc_desc(sA + kk * 256, 128, 1024);
        const uint64_t bd = tc_desc(sB + kk * 256, 128, 1024);
        const uint32_t acc = (kt | kk) != 0 ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&mbar[kt % kTcStages]))
          : "memory");
    }
    issued = kt + 1;
    // refill the stage read by chunk kt - 1 with chunk kt + kTcStages - 1
    const int nc = kt + kTcStages - 1;
    if (nc < nk) {
      if (kt >= 1 && !tc_wait(&mbar[(kt - 1) % kTcStages], ((kt - 1) / kTcStages) & 1)) ok = 0;
      if (ok) load(nc);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  // the last commit covers every MMA issued before it
  if (issued > 0 && !tc_wait(&mbar[(issued - 1) % kTcStages], ((issued - 1) / kTcStages) & 1))
    ok = 0;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  ok = __syncthreads_and(ok);
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows); warps 0-3 take
    // the even 16-column chunks, warps 4-7 the odd ones
    const int quarter = warp & 3, half = warp >> 2;
    const int64_t m = m0 + quarter * 32 + lane;
    const int32_t *idrow = nullptr;
    if (EPI == EPI_SCATTER_F64 && m < g.M) {
      const int64_t em = g.order ? g.order[m] : m;
      idrow = chk(bs_pred_index(em, g.M), BS_CHK_PREC_ENTRY) ? g.ids + em * g.np : nullptr;
    }
    for (int c0 = half * 16; c0 < npad; c0 += 32) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (m < g.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (c0 + j < nt) gemm_store<EPI>(g, m, n, __uint_as_float(v[j]), idrow);
        }
      }
    }
  } else if (tid == 0 && err) {
    atomicExch(err, 2);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols)
                 : "memory");
}

bool gemm_tc_supported(int epi, const GemmArgs &a) {
  return g_gemm_engine == 1 && a.K % 8 == 0 && a.K >= 8 && a.lda % 8 == 0 &&
         a.ldb % 8 == 0 && ((uintptr_t)a.A % 16) == 0 && ((uintptr_t)a.B % 16) == 0 &&
         epi != EPI_MASK_BF16;
}

template <int EPI>
static int launch_tc(const GemmArgs &a, int *err, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_gemm_tc<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tc_smem_bytes(kTcMaxN));
  });
  if (attr_err != cudaSuccess)
    return fail(BS_ERR_CUDA, "tcgen05 gemm: shared memory attribute: %s",
                cudaGetErrorString(attr_err));
  const int64_t gx = (a.M + kTcM - 1) / kTcM;
  const int gy = (a.N + kTcMaxN - 1) / kTcMaxN;
  const int ncol = a.N < kTcMaxN ? a.N : kTcMaxN;  // the widest tile
  k_gemm_tc<EPI><<<dim3((unsigned)gx, (unsigned)gy), kTcThreads, tc_smem_bytes((ncol + 15) & ~15),
                   s>>>(a, err);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

int launch_gemm_tc(int epi, const GemmArgs &a, int *err, cudaStream_t s) {
  switch (epi) {
    case EPI_F32: return launch_tc<EPI_F32>(a, err, s);
    case EPI_HIDDEN: return launch_tc<EPI_HIDDEN>(a, err, s);
    case EPI_SCALE_F64: return launch_tc<EPI_SCALE_F64>(a, err, s);
    case EPI_SCATTER_F64: return launch_tc<EPI_SCATTER_F64>(a, err, s);
    default: return fail(BS_ERR_ARG, "tcgen05 gemm: unsupported epilogue");
  }
}

}  // namespace bs

extern "C" int bs_gemm_engine(int32_t engine) {
  const int prev = bs::g_gemm_engine;
  if (engine == 0 || engine == 1) bs::g_gemm_engine = engine;
  return prev;
}
