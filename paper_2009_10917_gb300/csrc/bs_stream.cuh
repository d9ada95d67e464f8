// bs_stream.cuh -- BS1-BS5 kernels (Table 1), shared by the stand-alone C ABI
// entry points and the CG solvers.
//
// Design (GB300): grid-stride persistent blocks sized to a multiple of the SM
// count; 128-bit vector loads/stores (double2 / float4) with U independent
// vectors in flight per thread; streaming cache hints.  Reductions finish in
// the same launch: shuffle tree -> block -> last-block-done combine of the
// per-block partials in block-index order, so the result is deterministic.
// FP32 reductions carry each product and the running sum as unevaluated
// float pairs (error-free TwoProduct by fmaf, TwoSum), which keeps FP64-class
// accuracy on the FP32 pipes instead of GB300's narrow FP64 pipe.
#pragma once

#include "bs_internal.cuh"

namespace bs {

// A scalar that is either a value or read from device memory at run time.
template <typename T>
struct Scalar {
  T value;
  const T *ptr;
  __device__ __forceinline__ T get() const { return ptr ? *ptr : value; }
};

template <typename T> struct VecOf;
template <> struct VecOf<double> { using type = double2; static constexpr int W = 2; };
template <> struct VecOf<float> { using type = float4; static constexpr int W = 4; };

// Element access helpers for the vector types.
__device__ __forceinline__ double &vel(double2 &v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ float &vel(float4 &v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Split of [0, n) into a scalar head (to reach 16-byte alignment), a vector
// body and a scalar tail.  `vec` is false when the operands cannot share one
// alignment; then everything is scalar.
struct Split {
  int64_t head;   // scalar elements before the body
  int64_t nvec;   // vectors in the body
  int64_t tail0;  // first tail element
  int64_t n;
};

template <typename T>
inline Split make_split(int64_t n, const void *const *ptrs, int nptr) {
  constexpr int W = VecOf<T>::W;
  Split s{0, 0, 0, n};
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(ptrs[0]);
  bool same = true;
  for (int i = 1; i < nptr; ++i)
    same = same && ((reinterpret_cast<uintptr_t>(ptrs[i]) & 15u) == (a0 & 15u));
  if (!same || (a0 % sizeof(T)) != 0) {  // scalar only
    s.head = n;
    s.nvec = 0;
    s.tail0 = n;
    return s;
  }
  int64_t head = (int64_t)(((16u - (a0 & 15u)) & 15u) / sizeof(T));
  if (head > n) head = n;
  s.head = head;
  s.nvec = (n - head) / W;
  s.tail0 = head + s.nvec * W;
  return s;
}

// Float-float accumulation (Dekker/Knuth error-free transformations).
struct FF {
  float hi, lo;
};
__device__ __forceinline__ void ff_add_prod(FF &acc, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);       // a*b = p + e exactly
  const float s = acc.hi + p;           // TwoSum(acc.hi, p)
  const float bp = s - acc.hi;
  const float err = (acc.hi - (s - bp)) + (p - bp);
  acc.hi = s;
  acc.lo = acc.lo + (err + e);
}
__device__ __forceinline__ double ff_value(const FF &a) {
  return (double)a.hi + (double)a.lo;
}

// State the CG kernels share on the device.
struct CgState {
  double rr;      // r_j . r_j (or r.r of the latest update)
  double rz;      // r_j . z_j (preconditioned variants)
  double pAp;     // p . Ap
  double alpha;   // rr / pAp (or rz / pAp)
  double beta;    // ratio for the search direction update
  double eps;     // stop when rr <= eps
  double bb;      // b . b
  float alpha_f;  // alpha and -alpha rounded to float (FP32 inner solves)
  float beta_f;
  int iter;       // completed iterations
  int maxit;      // stop after this many iterations
  int fixed;      // 1: ignore eps
  int done;       // 0 running; 1 converged; 2 breakdown; 3 iteration limit
  int fallback;   // learned FPCG: 1 if this iteration's correction was rejected
  int nfallback;  // learned FPCG: corrections rejected so far
  double *hist;   // optional [3*(maxit+1)] alpha, beta, rr per iteration
  double rr_next; // block-Jacobi PCG: r.r and the Jacobi part of r.z of the
  double rz_next; // update, held until the interior blocks are solved
};

__device__ __forceinline__ bool cg_halted(const CgState *st) {
  return st != nullptr && *((volatile const int *)&st->done) != 0;
}

// The end of a CG iteration (Algorithm 1, steps 10-11 bookkeeping): record
// alpha, beta and r.r in the optional history, take beta and the new r.r,
// count the iteration and set the stop flag.
__device__ __forceinline__ void cg_advance(CgState *st, double rr_new, double beta) {
  const int j = st->iter;
  if (st->hist) {
    st->hist[3 * j] = st->alpha;
    st->hist[3 * j + 1] = beta;
    st->hist[3 * j + 2] = rr_new;
  }
  st->beta = beta;
  st->beta_f = (float)beta;
  st->rr = rr_new;
  st->iter = j + 1;
  if (!isfinite(rr_new) || !isfinite(beta))
    st->done = 2;
  else if (!st->fixed && rr_new <= st->eps)
    st->done = 1;
  else if (j + 1 >= st->maxit)
    st->done = 3;
}

}  // namespace bs

namespace bs {

// ------------------------------------------------------------ occupancy

// Resident blocks per SM for a kernel on the current device (cached).
template <typename K>
int blocks_per_sm(K kernel, int block) {
  return occupancy_blocks(reinterpret_cast<const void *>(kernel), block);
}

// Explicit fused multiply-add for either precision.
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// ------------------------------------------------------------ accumulators

template <typename T> struct Acc;
template <> struct Acc<double> {
  double a = 0.0;
  __device__ __forceinline__ void add(double x, double y) { a = fmaT(x, y, a); }
  __device__ __forceinline__ void merge(const Acc &o) { a = a + o.a; }
  __device__ __forceinline__ double value() const { return a; }
};
template <> struct Acc<float> {
  FF f{0.f, 0.f};
  __device__ __forceinline__ void add(float x, float y) { ff_add_prod(f, x, y); }
  __device__ __forceinline__ void merge(const Acc &o) {
    // TwoSum of the high parts, low parts added
    const float s = f.hi + o.f.hi;
    const float bp = s - f.hi;
    const float err = (f.hi - (s - bp)) + (o.f.hi - bp);
    f.hi = s;
    f.lo = f.lo + (err + o.f.lo);
  }
  __device__ __forceinline__ double value() const { return ff_value(f); }
};

// ------------------------------------------------------------ epilogues

struct EpStore {  // d_out[0] = total
  double *out;
  __device__ __forceinline__ void operator()(double s) const { out[0] = s; }
};
struct EpNorm {  // d_out[0] = total, d_out[1] = sqrt(total)
  double *out;
  __device__ __forceinline__ void operator()(double s) const {
    out[0] = s;
    out[1] = sqrt(s);
  }
};

// ------------------------------------------------------------ BS1 copy

template <typename T, int U>
__global__ void __launch_bounds__(kStreamBlock)
    k_copy(Split sp, const T *__restrict__ x, T *__restrict__ y) {
  using V = typename VecOf<T>::type;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const V *xv = reinterpret_cast<const V *>(x + sp.head);
  V *yv = reinterpret_cast<V *>(y + sp.head);
  int64_t i = tid;
  for (; i + (U - 1) * nth < sp.nvec; i += U * nth) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = ld_stream(xv + i + u * nth);
#pragma unroll
    for (int u = 0; u < U; ++u) st_stream(yv + i + u * nth, v[u]);
  }
  for (; i < sp.nvec; i += nth) st_stream(yv + i, ld_stream(xv + i));
  for (int64_t j = tid; j < sp.head; j += nth) y[j] = x[j];
  for (int64_t j = sp.tail0 + tid; j < sp.n; j += nth) y[j] = x[j];
}

template <typename T>
int launch_copy(int64_t n, const T *x, T *y, cudaStream_t s) {
  constexpr int U = 4;
  const void *ptrs[2] = {x, y};
  Split sp = make_split<T>(n, ptrs, 2);
  auto kern = k_copy<T, U>;
  const int64_t work = sp.nvec > 0 ? sp.nvec : n;
  const int grid = stream_grid(work, U, kStreamBlock, blocks_per_sm(kern, kStreamBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  kern<<<grid, kStreamBlock, 0, s>>>(sp, x, y);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// ------------------------------------------------------------ BS2 axpy

// y = fma(alpha, x, beta*y); with BETA1 the product 1*y == y is skipped.
template <typename T, int U, bool BETA1>
__global__ void __launch_bounds__(kStreamBlock)
    k_axpy(Split sp, Scalar<T> alpha_s, const T *__restrict__ x, Scalar<T> beta_s,
           T *__restrict__ y, const CgState *st) {
  using V = typename VecOf<T>::type;
  constexpr int W = VecOf<T>::W;
  if (cg_halted(st)) return;
  const T alpha = alpha_s.get();
  const T beta = beta_s.get();
  auto f = [&](T xv, T yv) -> T {
    if (BETA1) return fmaT(alpha, xv, yv);
    return fmaT(alpha, xv, beta * yv);
  };
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const V *xv = reinterpret_cast<const V *>(x + sp.head);
  V *yv = reinterpret_cast<V *>(y + sp.head);
  int64_t i = tid;
  for (; i + (U - 1) * nth < sp.nvec; i += U * nth) {
    V a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a[u] = ld_stream(xv + i + u * nth);
      b[u] = ld_stream(yv + i + u * nth);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int k = 0; k < W; ++k) vel(b[u], k) = f(vel(a[u], k), vel(b[u], k));
      st_stream(yv + i + u * nth, b[u]);
    }
  }
  for (; i < sp.nvec; i += nth) {
    V a = ld_stream(xv + i), b = ld_stream(yv + i);
#pragma unroll
    for (int k = 0; k < W; ++k) vel(b, k) = f(vel(a, k), vel(b, k));
    st_stream(yv + i, b);
  }
  for (int64_t j = tid; j < sp.head; j += nth) y[j] = f(x[j], y[j]);
  for (int64_t j = sp.tail0 + tid; j < sp.n; j += nth) y[j] = f(x[j], y[j]);
}

template <typename T>
int launch_axpy(int64_t n, Scalar<T> alpha, const T *x, Scalar<T> beta, T *y,
                const CgState *st, cudaStream_t s) {
  constexpr int U = 4;
  const void *ptrs[2] = {x, y};
  Split sp = make_split<T>(n, ptrs, 2);
  const bool beta1 = beta.ptr == nullptr && beta.value == T(1);
  auto kern = beta1 ? k_axpy<T, U, true> : k_axpy<T, U, false>;
  const int64_t work = sp.nvec > 0 ? sp.nvec : n;
  const int grid = stream_grid(work, U, kStreamBlock, blocks_per_sm(kern, kStreamBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  kern<<<grid, kStreamBlock, 0, s>>>(sp, alpha, x, beta, y, st);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// ------------------------------------------------------------ BS3/BS4 norm, dot

// Sum of x[i]*y[i] (SELF: y = x, read once), one launch.
template <typename T, int U, bool SELF, class Ep>
__global__ void __launch_bounds__(kReduceBlock)
    k_dot(Split sp, const T *__restrict__ x, const T *__restrict__ y, double *partials,
          unsigned int *counter, Ep ep, const CgState *st) {
  using V = typename VecOf<T>::type;
  constexpr int W = VecOf<T>::W;
  if (cg_halted(st)) return;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const V *xv = reinterpret_cast<const V *>(x + sp.head);
  const V *yv = reinterpret_cast<const V *>(y + sp.head);
  Acc<T> acc[U];
  int64_t i = tid;
  for (; i + (U - 1) * nth < sp.nvec; i += U * nth) {
    V a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a[u] = ld_stream(xv + i + u * nth);
      if (!SELF) b[u] = ld_stream(yv + i + u * nth);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < W; ++k)
        acc[u].add(vel(a[u], k), SELF ? vel(a[u], k) : vel(b[u], k));
  }
  for (; i < sp.nvec; i += nth) {
    V a = ld_stream(xv + i);
    V b = SELF ? a : ld_stream(yv + i);
#pragma unroll
    for (int k = 0; k < W; ++k) acc[0].add(vel(a, k), vel(b, k));
  }
  for (int64_t j = tid; j < sp.head; j += nth) acc[0].add(x[j], SELF ? x[j] : y[j]);
  for (int64_t j = sp.tail0 + tid; j < sp.n; j += nth) acc[0].add(x[j], SELF ? x[j] : y[j]);
#pragma unroll
  for (int u = 1; u < U; ++u) acc[0].merge(acc[u]);
  const double part = block_sum<kReduceBlock>(acc[0].value());
  double total;
  if (grid_combine<kReduceBlock>(part, partials, counter, &total) && threadIdx.x == 0)
    ep(total);
}

template <typename T, bool SELF, class Ep>
int launch_dot(int64_t n, const T *x, const T *y, double *partials, unsigned int *counter,
               Ep ep, const CgState *st, cudaStream_t s) {
  constexpr int U = 4;
  const void *ptrs[2] = {x, y};
  Split sp = make_split<T>(n, ptrs, SELF ? 1 : 2);
  auto kern = k_dot<T, U, SELF, Ep>;
  const int64_t work = sp.nvec > 0 ? sp.nvec : n;
  int grid = stream_grid(work, U, kReduceBlock, blocks_per_sm(kern, kReduceBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  if (grid > kMaxPartials) grid = kMaxPartials;
  kern<<<grid, kReduceBlock, 0, s>>>(sp, x, y, partials, counter, ep, st);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// ------------------------------------------------------------ BS3 norm, FP64

// On GB300 one DFMA per 8 bytes read is more than the FP64 pipe sustains, so
// the FP64 norm moves half of the squares onto the FP32 pipes.  An element x
// with 2^-30 <= |x| < 2^31 is split exactly by integer operations into
// h = x truncated to 24 significant bits (a float) and l = the remaining 29
// bits rounded to a float (relative error of h + l below 2^-47); then
// x^2 = h^2 + (fma(h, h, -h^2) + 2 h l + l^2), the first term exact.  These
// pairs accumulate as an unevaluated float pair for 16 elements, then the
// chunk joins a double accumulator.  Every other element (and any element
// outside the window: zeros, subnormals, huge values) takes a DFMA.
struct SqAcc {
  FF f{0.f, 0.f};
  double d = 0.0;    // FP64 squares and flushed float-pair chunks
  double dd = 0.0;   // second FP64 chain for ILP
  __device__ __forceinline__ void add_dfma(double x) { dd = fma(x, x, dd); }
  __device__ __forceinline__ void add_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned E = (hw >> 20) & 0x7ffu;
    if (E - 993u > 60u) {  // outside [2^-30, 2^31)
      d = fma(x, x, d);
      return;
    }
    const unsigned sign = hw & 0x80000000u;
    const float h = __uint_as_float(sign | ((E - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    // l = the low 29 bits r, rounded to a multiple of 2^6, times 2^(E - 1075):
    // with base = 2^(E - 1046) as a float, the bit pattern base + rr is
    // base * (1 + rr / 2^23), so subtracting base leaves rr * 2^(E - 1069)
    // exactly (rr = 2^23 carries into the exponent and still gives rr * 2^..).
    // Integer and FP32 operations only: conversion instructions share GB300's
    // narrow FP64 pipe.
    const unsigned rr = ((lw & 0x1fffffffu) + 32u) >> 6;
    const unsigned base = (E - 919u) << 23;
    const float l = __uint_as_float(
        __float_as_uint(__uint_as_float(base + rr) - __uint_as_float(base)) | sign);
    const float p = h * h;
    const float t = fmaf(h + h, l, fmaf(l, l, fmaf(h, h, -p)));
    const float s = f.hi + p;  // TwoSum(f.hi, p)
    const float bp = s - f.hi;
    const float err = (f.hi - (s - bp)) + (p - bp);
    f.hi = s;
    f.lo = f.lo + (err + t);
  }
  // A normal or zero float as a double, by assembling the bits (no
  // conversion instruction).  Subnormal floats (never produced here: the
  // window keeps every term above 2^-120) would flush to zero.
  static __device__ __forceinline__ double widen(float v) {
    const unsigned u = __float_as_uint(v);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  __device__ __forceinline__ void flush() {
    d = d + (widen(f.hi) + widen(f.lo));
    f.hi = 0.f;
    f.lo = 0.f;
  }
  __device__ __forceinline__ double value() {
    flush();
    return d + dd;
  }
};

template <int U, class Ep>
__global__ void __launch_bounds__(kReduceBlock)
    k_norm_split(Split sp, const double *__restrict__ x, double *partials, unsigned int *counter,
                 Ep ep) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const double2 *xv = reinterpret_cast<const double2 *>(x + sp.head);
  SqAcc acc;
  int64_t i = tid;
  int chunk = 0;
  for (; i + (U - 1) * nth < sp.nvec; i += U * nth) {
    double2 a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = ld_stream(xv + i + u * nth);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      acc.add_split(a[u].x);
      acc.add_dfma(a[u].y);
    }
    if (++chunk == 16 / U) {
      acc.flush();
      chunk = 0;
    }
  }
  for (; i < sp.nvec; i += nth) {
    const double2 a = ld_stream(xv + i);
    acc.add_dfma(a.x);
    acc.add_dfma(a.y);
  }
  for (int64_t j = tid; j < sp.head; j += nth) acc.add_dfma(x[j]);
  for (int64_t j = sp.tail0 + tid; j < sp.n; j += nth) acc.add_dfma(x[j]);
  const double part = block_sum<kReduceBlock>(acc.value());
  double total;
  if (grid_combine<kReduceBlock>(part, partials, counter, &total) && threadIdx.x == 0) ep(total);
}

template <class Ep>
int launch_norm_split(int64_t n, const double *x, double *partials, unsigned int *counter, Ep ep,
                      cudaStream_t s) {
  constexpr int U = 4;
  const void *ptrs[1] = {x};
  Split sp = make_split<double>(n, ptrs, 1);
  auto kern = k_norm_split<U, Ep>;
  const int64_t work = sp.nvec > 0 ? sp.nvec : n;
  int grid = stream_grid(work, U, kReduceBlock, blocks_per_sm(kern, kReduceBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  if (grid > kMaxPartials) grid = kMaxPartials;
  kern<<<grid, kReduceBlock, 0, s>>>(sp, x, partials, counter, ep);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

// ------------------------------------------------------------ BS5 fused CG update

// x = fma(alpha, p, x); r = fma(-alpha, Ap, r); total = sum r^2; one pass.
template <typename T, int U, class Ep>
__global__ void __launch_bounds__(kReduceBlock)
    k_cg_update(Split sp, Scalar<T> alpha_s, const T *__restrict__ p, const T *__restrict__ Ap,
                T *__restrict__ x, T *__restrict__ r, double *partials, unsigned int *counter,
                Ep ep, const CgState *st) {
  using V = typename VecOf<T>::type;
  constexpr int W = VecOf<T>::W;
  if (cg_halted(st)) return;
  const T alpha = alpha_s.get();
  const T nalpha = -alpha;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const V *pv = reinterpret_cast<const V *>(p + sp.head);
  const V *Apv = reinterpret_cast<const V *>(Ap + sp.head);
  V *xv = reinterpret_cast<V *>(x + sp.head);
  V *rv = reinterpret_cast<V *>(r + sp.head);
  Acc<T> acc[U];
  int64_t i = tid;
  for (; i + (U - 1) * nth < sp.nvec; i += U * nth) {
    V a[U], b[U], c[U], d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a[u] = ld_stream(pv + i + u * nth);
      b[u] = ld_stream(Apv + i + u * nth);
      c[u] = ld_stream(xv + i + u * nth);
      d[u] = ld_stream(rv + i + u * nth);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int k = 0; k < W; ++k) {
        vel(c[u], k) = fmaT(alpha, vel(a[u], k), vel(c[u], k));
        vel(d[u], k) = fmaT(nalpha, vel(b[u], k), vel(d[u], k));
        acc[u].add(vel(d[u], k), vel(d[u], k));
      }
      st_stream(xv + i + u * nth, c[u]);
      st_stream(rv + i + u * nth, d[u]);
    }
  }
  for (; i < sp.nvec; i += nth) {
    V a = ld_stream(pv + i), b = ld_stream(Apv + i), c = ld_stream(xv + i), d = ld_stream(rv + i);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      vel(c, k) = fmaT(alpha, vel(a, k), vel(c, k));
      vel(d, k) = fmaT(nalpha, vel(b, k), vel(d, k));
      acc[0].add(vel(d, k), vel(d, k));
    }
    st_stream(xv + i, c);
    st_stream(rv + i, d);
  }
  auto scalar = [&](int64_t j) {
    x[j] = fmaT(alpha, p[j], x[j]);
    const T rj = fmaT(nalpha, Ap[j], r[j]);
    r[j] = rj;
    acc[0].add(rj, rj);
  };
  for (int64_t j = tid; j < sp.head; j += nth) scalar(j);
  for (int64_t j = sp.tail0 + tid; j < sp.n; j += nth) scalar(j);
#pragma unroll
  for (int u = 1; u < U; ++u) acc[0].merge(acc[u]);
  const double part = block_sum<kReduceBlock>(acc[0].value());
  double total;
  if (grid_combine<kReduceBlock>(part, partials, counter, &total) && threadIdx.x == 0)
    ep(total);
}

template <typename T, class Ep>
int launch_cg_update(int64_t n, Scalar<T> alpha, const T *p, const T *Ap, T *x, T *r,
                     double *partials, unsigned int *counter, Ep ep, const CgState *st,
                     cudaStream_t s) {
  constexpr int U = 2;
  const void *ptrs[4] = {p, Ap, x, r};
  Split sp = make_split<T>(n, ptrs, 4);
  auto kern = k_cg_update<T, U, Ep>;
  const int64_t work = sp.nvec > 0 ? sp.nvec : n;
  int grid = stream_grid(work, U, kReduceBlock, blocks_per_sm(kern, kReduceBlock));
  if (grid < 1) return fail(BS_ERR_CUDA, "no device");
  if (grid > kMaxPartials) grid = kMaxPartials;
  kern<<<grid, kReduceBlock, 0, s>>>(sp, alpha, p, Ap, x, r, partials, counter, ep, st);
  BS_LAUNCH_CHECK();
  return BS_OK;
}

}  // namespace bs
