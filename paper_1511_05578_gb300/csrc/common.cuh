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
__host__ __device__ __forceinline__ double parity_sign(int k) { return (k & 1) ? -1.0 : 1.0; }

// Record a launch of one of our kernels (host side).
void count_launch();
// Check the last launch; on failure store a message and return false.
bool launch_ok(const char* what);

}  // namespace crv
