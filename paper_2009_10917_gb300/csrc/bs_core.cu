// bs_core.cu -- status strings, thread-local error detail, device queries and
// the reduction workspace.
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "bs_internal.cuh"

namespace bs {

static thread_local char t_err[512] = "";

int fail(int status, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_err, sizeof(t_err), fmt, ap);
  va_end(ap);
  return status;
}

void clear_error() { t_err[0] = '\0'; }

int device_info(DeviceInfo *out) {
  static std::mutex mu;
  static DeviceInfo cache[64];
  int dev = 0;
  BS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(BS_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (cache[dev].device != dev) {
    DeviceInfo d;
    d.device = dev;
    BS_CUDA_TRY(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    BS_CUDA_TRY(cudaDeviceGetAttribute(&d.max_threads_sm,
                                       cudaDevAttrMaxThreadsPerMultiProcessor, dev));
    cache[dev] = d;
  }
  *out = cache[dev];
  return BS_OK;
}

int stream_grid(int64_t work, int per_thread, int block, int blocks_per_sm) {
  DeviceInfo d;
  if (device_info(&d) != BS_OK) return 0;
  const int64_t full = (int64_t)d.sms * blocks_per_sm;
  const int64_t per_block = (int64_t)block * per_thread;
  int64_t need = (work + per_block - 1) / per_block;
  if (need < 1) need = 1;
  return (int)(need < full ? need : full);
}

int occupancy_blocks(const void *kernel, int block) {
  static std::mutex mu;
  static std::map<std::tuple<const void *, int, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_tuple(kernel, block, dev);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, block, 0) != cudaSuccess || b < 1)
    b = 1;
  cache[key] = b;
  return b;
}

// The check-word readers of all translation units (checked build; empty in
// the default build).
static std::mutex g_check_mu;
static std::vector<int (*)(unsigned int *)> &check_readers() {
  static std::vector<int (*)(unsigned int *)> v;
  return v;
}

int register_check_word(int (*read_and_clear)(unsigned int *)) {
  std::lock_guard<std::mutex> lock(g_check_mu);
  check_readers().push_back(read_and_clear);
  return (int)check_readers().size();
}

[[maybe_unused]] static const char *check_code_name(unsigned int code) {
  switch (code) {
    case BS_CHK_SCATTER_ENTRY: return "scatter: map entry >= N_G";
    case BS_CHK_GATHER_TILE: return "gather: tile bounds outside the CSR";
    case BS_CHK_GATHER_ROW: return "gather: row bounds outside [0, nnz]";
    case BS_CHK_GATHER_COL: return "gather: column >= N_L";
    case BS_CHK_GATHER_CHUNK: return "pipelined gather: chunk id outside q_L";
    case BS_CHK_GATHER_STAGED: return "pipelined gather: offset outside the staged tile";
    case BS_CHK_OP_ENTRY: return "element operator: map entry out of range";
    case BS_CHK_PREC_ENTRY: return "preconditioner or network epilogue: map entry out of range";
    case BS_CHK_ROWS: return "multi-rank rows: index out of range";
    case BS_CHK_BATCH: return "batched solver: index out of range";
    default: return "unknown check";
  }
}

int occupancy_blocks_smem(const void *kernel, int block, int smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void *, int, int, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_tuple(kernel, block, smem, dev);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int b = 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, block, smem) != cudaSuccess)
    b = 0;
  cache[key] = b;
  return b;
}

}  // namespace bs

extern "C" {

const char *bs_error_string(int status) {
  switch (status) {
    case BS_OK: return "success";
    case BS_ERR_ARG: return "invalid argument";
    case BS_ERR_CUDA: return "CUDA runtime error";
    case BS_ERR_TIMEOUT: return "device-side wait timed out";
    case BS_ERR_BREAKDOWN: return "CG breakdown (p.Ap <= 0 or not finite)";
    case BS_ERR_NOT_CONVERGED: return "iteration limit reached before tolerance";
    case BS_ERR_DEVICE_CHECK: return "device-side check failed";
    case BS_ERR_ALLOC: return "allocation failed";
    default: return "unknown status";
  }
}

const char *bs_last_error(void) { return bs::t_err; }

int bs_version(void) { return 10000; }

int bs_check_enabled(void) { return BS_CHECK ? 1 : 0; }

int bs_check_device(void) {
#if !BS_CHECK
  return BS_OK;
#else
  BS_CUDA_TRY(cudaDeviceSynchronize());
  unsigned int first = 0;
  int nfail = 0;
  std::lock_guard<std::mutex> lock(bs::g_check_mu);
  for (auto rd : bs::check_readers()) {
    unsigned int w = 0;
    if (rd(&w) != 0) return bs::fail(BS_ERR_CUDA, "bs_check_device: reading a check word");
    if (w) {
      ++nfail;
      if (!first) first = w;
    }
  }
  if (first)
    return bs::fail(BS_ERR_DEVICE_CHECK, "device check %u (%s) failed in %d unit(s)", first,
                    bs::check_code_name(first), nfail);
  return BS_OK;
#endif
}

int bs_workspace_create(bs_workspace **ws) {
  BS_ARG(ws != nullptr, "bs_workspace_create: ws is NULL");
  *ws = nullptr;
  bs_workspace *w = (bs_workspace *)calloc(1, sizeof(bs_workspace));
  if (!w) return bs::fail(BS_ERR_ALLOC, "bs_workspace_create: host allocation");
  cudaError_t e = cudaGetDevice(&w->device);
  void *mem = nullptr;
  if (e == cudaSuccess)
    e = cudaMalloc(&mem, bs::kMaxPartials * sizeof(double) + 256);
  if (e == cudaSuccess) e = cudaMemset(mem, 0, bs::kMaxPartials * sizeof(double) + 256);
  if (e != cudaSuccess) {
    if (mem) cudaFree(mem);
    free(w);
    return bs::fail(BS_ERR_CUDA, "bs_workspace_create: %s", cudaGetErrorString(e));
  }
  w->partials = (double *)mem;
  w->counter = (unsigned int *)((char *)mem + bs::kMaxPartials * sizeof(double));
  *ws = w;
  return BS_OK;
}

int bs_workspace_destroy(bs_workspace *ws) {
  if (!ws) return BS_OK;
  cudaError_t e = cudaFree(ws->partials);
  free(ws);
  if (e != cudaSuccess)
    return bs::fail(BS_ERR_CUDA, "bs_workspace_destroy: %s", cudaGetErrorString(e));
  return BS_OK;
}

}  // extern "C"
