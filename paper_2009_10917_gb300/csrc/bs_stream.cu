// bs_stream.cu -- C ABI entry points of BS1-BS5 (Table 1) and their FP32
// twins.  Kernels live in bs_stream.cuh.
#include "bs_stream.cuh"

namespace bs {

static int check_ws(const bs_workspace *ws, const char *fn) {
  if (!ws) return fail(BS_ERR_ARG, "%s: workspace is NULL", fn);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ws->device)
    return fail(BS_ERR_ARG, "%s: workspace belongs to device %d, current is %d", fn,
                ws->device, dev);
  return BS_OK;
}

template <typename T>
static int do_copy(int64_t n, const T *x, T *y, void *stream, const char *fn) {
  BS_ARG(n >= 0, "%s: n < 0", fn);
  if (n == 0) return BS_OK;
  BS_ARG(x && y, "%s: NULL vector", fn);
  return launch_copy<T>(n, x, y, as_stream(stream));
}

template <typename T>
static int do_axpy(int64_t n, T alpha, const T *x, T beta, T *y, void *stream,
                   const char *fn) {
  BS_ARG(n >= 0, "%s: n < 0", fn);
  if (n == 0) return BS_OK;
  BS_ARG(x && y, "%s: NULL vector", fn);
  BS_ARG(x + n <= y || y + n <= x, "%s: x and y overlap", fn);
  return launch_axpy<T>(n, Scalar<T>{alpha, nullptr}, x, Scalar<T>{beta, nullptr}, y, nullptr,
                        as_stream(stream));
}

template <typename T, bool SELF, class Ep>
static int do_dot(int64_t n, const T *x, const T *y, Ep ep, double *out, bs_workspace *ws,
                  void *stream, const char *fn) {
  BS_ARG(n >= 0, "%s: n < 0", fn);
  BS_ARG(out != nullptr, "%s: NULL output", fn);
  if (int rc = check_ws(ws, fn)) return rc;
  if (n > 0) BS_ARG(x && y, "%s: NULL vector", fn);
  // n == 0 runs the kernel on an empty range: one block writes the zero sum.
  return launch_dot<T, SELF, Ep>(n, x, y, ws->partials, ws->counter, ep, nullptr,
                                 as_stream(stream));
}

template <typename T>
static int do_cg_update(int64_t n, T alpha, const T *p, const T *Ap, T *x, T *r, double *d_rr,
                        bs_workspace *ws, void *stream, const char *fn) {
  BS_ARG(n >= 0, "%s: n < 0", fn);
  BS_ARG(d_rr != nullptr, "%s: NULL output", fn);
  if (int rc = check_ws(ws, fn)) return rc;
  if (n > 0) BS_ARG(p && Ap && x && r, "%s: NULL vector", fn);
  return launch_cg_update<T, EpStore>(n, Scalar<T>{alpha, nullptr}, p, Ap, x, r, ws->partials,
                                      ws->counter, EpStore{d_rr}, nullptr, as_stream(stream));
}

}  // namespace bs

using namespace bs;

extern "C" {

int bs_copy(int64_t n, const double *x, double *y, void *stream) {
  return do_copy<double>(n, x, y, stream, "bs_copy");
}
int bs_copy_f32(int64_t n, const float *x, float *y, void *stream) {
  return do_copy<float>(n, x, y, stream, "bs_copy_f32");
}

int bs_axpy(int64_t n, double alpha, const double *x, double beta, double *y, void *stream) {
  return do_axpy<double>(n, alpha, x, beta, y, stream, "bs_axpy");
}
int bs_axpy_f32(int64_t n, float alpha, const float *x, float beta, float *y, void *stream) {
  return do_axpy<float>(n, alpha, x, beta, y, stream, "bs_axpy_f32");
}

int bs_norm(int64_t n, const double *x, double *d_out, bs_workspace *ws, void *stream) {
  BS_ARG(n >= 0, "bs_norm: n < 0");
  BS_ARG(d_out != nullptr, "bs_norm: NULL output");
  if (int rc = check_ws(ws, "bs_norm")) return rc;
  if (n > 0) BS_ARG(x != nullptr, "bs_norm: NULL vector");
  return launch_norm_split(n, x, ws->partials, ws->counter, EpNorm{d_out}, as_stream(stream));
}
int bs_norm_f32(int64_t n, const float *x, double *d_out, bs_workspace *ws, void *stream) {
  return do_dot<float, true>(n, x, x, EpNorm{d_out}, d_out, ws, stream, "bs_norm_f32");
}

int bs_dot(int64_t n, const double *x, const double *y, double *d_out, bs_workspace *ws,
           void *stream) {
  return do_dot<double, false>(n, x, y, EpStore{d_out}, d_out, ws, stream, "bs_dot");
}
int bs_dot_f32(int64_t n, const float *x, const float *y, double *d_out, bs_workspace *ws,
               void *stream) {
  return do_dot<float, false>(n, x, y, EpStore{d_out}, d_out, ws, stream, "bs_dot_f32");
}

int bs_cg_update(int64_t n, double alpha, const double *p, const double *Ap, double *x,
                 double *r, double *d_rr, bs_workspace *ws, void *stream) {
  return do_cg_update<double>(n, alpha, p, Ap, x, r, d_rr, ws, stream, "bs_cg_update");
}
int bs_cg_update_f32(int64_t n, float alpha, const float *p, const float *Ap, float *x,
                     float *r, double *d_rr, bs_workspace *ws, void *stream) {
  return do_cg_update<float>(n, alpha, p, Ap, x, r, d_rr, ws, stream, "bs_cg_update_f32");
}

}  // extern "C"
