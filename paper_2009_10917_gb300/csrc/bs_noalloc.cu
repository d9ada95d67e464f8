// bs_noalloc.cu -- bs_dot_noalloc: the BS4 inner product with its reduction
// scratch in static device memory, for callers that cannot allocate device
// memory (they own all device memory through their own pool, or cannot
// afford the device-wide synchronisation of cudaMalloc/cudaFree).
//
// The scratch is one file-scope __device__ array: BS_NOALLOC_MAX_PARTIALS
// per-block partial sums followed by the arrival counter of the last-block-
// done combine.  Host code must not hand the array's name to a kernel: on the
// host it is only a stand-in symbol, not a device address.  Its device
// address is looked up once per device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "bs_stream.cuh"

namespace {

constexpr int kCap = BS_NOALLOC_MAX_PARTIALS;
constexpr int kMaxDevices = 64;

// [0, kCap): partials; [kCap]: arrival counter (as unsigned int); padding.
static __device__ __align__(256) double g_dot_scratch[kCap + 32];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_dot_scratch on the current device (looked up on the
// first call per device, with that device current).
int scratch_address(double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return bs::fail(BS_ERR_CUDA, "bs_dot_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return bs::fail(BS_ERR_ARG, "bs_dot_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dot_scratch);
    if (e != cudaSuccess || p == nullptr)
      return bs::fail(BS_ERR_CUDA, "bs_dot_noalloc: cudaGetSymbolAddress: %s",
                      cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return BS_OK;
}

}  // namespace

extern "C" int bs_dot_noalloc(int64_t n, const double *x, const double *y, double *d_out,
                              void *stream) {
  using namespace bs;
  BS_ARG(n >= 0, "bs_dot_noalloc: n < 0");
  BS_ARG(d_out != nullptr, "bs_dot_noalloc: NULL output");
  if (n > 0) BS_ARG(x && y, "bs_dot_noalloc: NULL vector");
  double *scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;
  constexpr int U = 4;
  const void *ptrs[2] = {x, y};
  const Split sp = make_split<double>(n, ptrs, 2);
  auto kern = k_dot<double, U, false, EpStore>;
  const int64_t work = sp.nvec > 0 ? sp.nvec : n;
  int grid = stream_grid(work, U, kReduceBlock, blocks_per_sm(kern, kReduceBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "bs_dot_noalloc: no device");
  // k_dot is grid-stride: a smaller grid covers any n, so the partials never
  // outgrow the static array (the workspace form clamps the same way)
  if (grid > kCap) grid = kCap;
  cudaStream_t s = as_stream(stream);
  unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + kCap);
  BS_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
  kern<<<grid, kReduceBlock, 0, s>>>(sp, x, y, scratch, counter, EpStore{d_out}, nullptr);
  BS_LAUNCH_CHECK();
  return BS_OK;
}
