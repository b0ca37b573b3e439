// Shared device/host helpers of libcrv: complex arithmetic, error plumbing,
// launch accounting.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace crv {

template <class T>
struct __align__(2 * sizeof(T)) cx {
  T re, im;
};

template <class T> __host__ __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.re = a; r.im = b; return r; }
template <class T> __host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <class T> __host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
// FP32 complex addition and subtraction on the device as one paired instruction each
// (add.rn.f32x2 / sub.rn.f32x2 of sm_100 and later: IEEE round-to-nearest per component,
// the same results as two scalar operations, half the issue slots).
__host__ __device__ __forceinline__ cx<float> operator+(cx<float> a, cx<float> b) {
#ifdef __CUDA_ARCH__
  uint64_t x, y, z;
  asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.re), "f"(a.im));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.re), "f"(b.im));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
  cx<float> r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.re), "=f"(r.im) : "l"(z));
  return r;
#else
  return mk(a.re + b.re, a.im + b.im);
#endif
}
__host__ __device__ __forceinline__ cx<float> operator-(cx<float> a, cx<float> b) {
#ifdef __CUDA_ARCH__
  uint64_t x, y, z;
  asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.re), "f"(a.im));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.re), "f"(b.im));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
  cx<float> r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.re), "=f"(r.im) : "l"(z));
  return r;
#else
  return mk(a.re - b.re, a.im - b.im);
#endif
}
template <class T> __host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T> __host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, T s) { return mk(a.re * s, a.im * s); }
template <class T> __host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return mk(a.re, -a.im); }
// multiply by i^k
template <class T> __host__ __device__ __forceinline__ cx<T> mul_ipow(cx<T> a, int k) {
  switch (k & 3) {
    case 0: return a;
    case 1: return mk(-a.im, a.re);
    case 2: return mk(-a.re, -a.im);
    default: return mk(a.im, -a.re);
  }
}
__host__ __device__ __forceinline__ int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

// Double-float: an unevaluated sum hi + lo of two FP32 values (|lo| <= ulp(hi)/2), about 48
// significant bits, with additions and multiplications in FP32 instructions (Knuth's two-sum
// and the FMA product error, then renormalised). The FP64 plans run their largest Wigner FFTs
// in it: GB300 issues FP32 at many times its FP64 rate. The error-free steps must not be fused
// into FMAs or reassociated: on the device they use the _rn intrinsics, which the compiler never
// contracts. (Host code only converts to and from double.)
struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ df(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ df(float x) : hi(x), lo(0.f) {}
  __host__ __device__ df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
#ifdef __CUDA_ARCH__
__device__ __forceinline__ df operator+(df a, df b) {
  const float s = __fadd_rn(a.hi, b.hi), bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));  // s + e = a.hi + b.hi
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df r;
  r.hi = __fadd_rn(s, e);
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
  return r;
}
__device__ __forceinline__ df operator-(df a) {
  df r;
  r.hi = -a.hi;
  r.lo = -a.lo;
  return r;
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // p + e = a.hi b.hi exactly
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df r;
  r.hi = __fadd_rn(p, e);
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, p));
  return r;
}
#endif

// Exact division of 32-bit unsigned n by a runtime constant d (1 <= d < 2^32) with a
// 64-bit reciprocal M = floor((2^64-1)/d) + 1: n / d = mulhi64(M, n) (Lemire et al.,
// "Faster remainder by direct computation", 2019).
struct FastDiv {
  uint32_t d = 1;
  uint64_t M = 0;
  FastDiv() = default;
  __host__ explicit FastDiv(uint32_t dd) : d(dd), M(~0ull / dd + 1) {}
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return d == 1 ? n : (uint32_t)__umul64hi(M, (uint64_t)n); }
  __device__ __forceinline__ uint32_t mod(uint32_t n) const { return n - div(n) * d; }
};
__host__ __device__ __forceinline__ double parity_sign(int k) { return (k & 1) ? -1.0 : 1.0; }

// Kernel kinds, for launch accounting and optional event timing.
enum KernelKind {
  K_DELTA = 0, K_SHT_CONTRACT, K_SHT_ROWS, K_BETA_SYNTH, K_BETA_QUAD, K_RING_INV_N, K_RING_INV_M,
  K_RING_FWD_G, K_RING_FWD_A, K_CONTRACT_A, K_CONTRACT_S, K_TC_A, K_TC_S, K_MISC, K_SHT_BETA, K_ROTATE, K_OZ_A, K_OZ_S, K_NKINDS
};
const char* kind_name(int k);

// Brackets one launch: records a start event on the stream if that kind is being
// timed; done() records the end event and counts the launch.
struct KTimer {
  int kind;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  KTimer(int kind, cudaStream_t s);
  void done();
};

// Record a launch of one of our kernels (host side).
void count_launch();
// Per-device launch facts, cached per device ordinal (thread-safe): the current device's
// SM count, and a kernel's dynamic shared-memory limit raised once on each device.
int device_sms();
bool func_attr_once(const void* kernel, int smem_bytes);
// Preferred shared-memory carveout of a kernel for `blocks` blocks of `bytes` each (once per
// device): the rest of the unified L1 stays cache.
void carveout_for(const void* kernel, size_t bytes, int blocks);
// Check the last launch; on failure store a message and return false.
bool launch_ok(const char* what);

}  // namespace crv
