// Shared-memory FFT engine for the odd lengths N = 2L_j - 1 of the MW / SO(3)
// grids (Eqs. nodes_alpha..nodes_gamma). A length-N DFT is done by Bluestein's
// chirp-z identity jk = (j^2 + k^2 - (k-j)^2)/2, which turns it into a cyclic
// convolution of length P = 2^p >= 2N-1, itself done by a Stockham radix-4/2
// power-of-two FFT in shared memory. One code path serves every length (the
// prime factors of 2L-1 reach 89 at L = 1024).
#pragma once
#include "common.cuh"

namespace crv {

// Device tables for one length N, one precision.
template <class T>
struct DftTab {
  int N = 0, P = 0;
  const cx<T>* tw = nullptr;      // [P]  e^{-2 pi i k / P}
  const cx<T>* chirp = nullptr;   // [N]  h_t = e^{-i pi t^2 / N}
  const cx<T>* khat_f = nullptr;  // [P]  FFT_P(conj h wrapped) / P   (forward DFT, sign -1)
  const cx<T>* khat_i = nullptr;  // [P]  FFT_P(h wrapped) / P        (inverse DFT, sign +1)
};

// Stockham autosort FFT of `nb` independent length-P transforms held back to
// back in x (each of length P); y is scratch of the same size. Returns the buffer
// holding the result (x or y). dir = -1 forward (e^{-i}), +1 inverse (no 1/P).
template <class T>
__device__ cx<T>* fft_pow2(cx<T>* x, cx<T>* y, int P, int nb, const cx<T>* __restrict__ tw, int dir) {
  const int tid = threadIdx.x, nth = blockDim.x;
  int Ns = 1;
  while (Ns < P) {
    const int R = (P / Ns >= 4) ? 4 : 2;
    const int nbf = P / R;             // butterflies per transform
    const int stride = P / (Ns * R);   // twiddle index step
    for (int t = tid; t < nb * nbf; t += nth) {
      const int b = t / nbf, j = t - b * nbf;
      const cx<T>* xb = x + (size_t)b * P;
      cx<T>* yb = y + (size_t)b * P;
      const int k = j & (Ns - 1);
      const int out = ((j - k) * R) + k;
      if (R == 4) {
        cx<T> v0 = xb[j], v1 = xb[j + nbf], v2 = xb[j + 2 * nbf], v3 = xb[j + 3 * nbf];
        if (Ns > 1) {
          cx<T> w1 = tw[k * stride], w2 = tw[2 * k * stride], w3 = tw[3 * k * stride];
          if (dir > 0) { w1 = conj(w1); w2 = conj(w2); w3 = conj(w3); }
          v1 = v1 * w1; v2 = v2 * w2; v3 = v3 * w3;
        }
        cx<T> a0 = v0 + v2, a1 = v0 - v2, a2 = v1 + v3, d = v1 - v3;
        cx<T> a3 = (dir < 0) ? mk(d.im, -d.re) : mk(-d.im, d.re);
        yb[out] = a0 + a2;
        yb[out + Ns] = a1 + a3;
        yb[out + 2 * Ns] = a0 - a2;
        yb[out + 3 * Ns] = a1 - a3;
      } else {
        cx<T> v0 = xb[j], v1 = xb[j + nbf];
        if (Ns > 1) {
          cx<T> w1 = tw[k * stride];
          if (dir > 0) w1 = conj(w1);
          v1 = v1 * w1;
        }
        yb[out] = v0 + v1;
        yb[out + Ns] = v0 - v1;
      }
    }
    __syncthreads();
    cx<T>* s = x; x = y; y = s;
    Ns *= R;
  }
  return x;
}

// Bluestein DFT of `nb` length-N sequences. On entry buf[b*P + j], j < N, holds
// x_j of sequence b (entries j >= N are ignored). On exit the returned pointer p
// has X_k at p[b*P + k], k < N, where X_k = sum_j x_j e^{sign 2 pi i j k / N}.
// buf and scr are shared-memory buffers of nb*P elements each.
template <class T>
__device__ cx<T>* dft_bluestein(cx<T>* buf, cx<T>* scr, int nb, const DftTab<T>& tb, int sign) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int N = tb.N, P = tb.P;
  // a_j = x_j h^sign_j, zero padded
  for (int t = tid; t < nb * P; t += nth) {
    const int j = t % P;
    cx<T> v = mk<T>(0, 0);
    if (j < N) {
      cx<T> h = tb.chirp[j];
      if (sign > 0) h = conj(h);
      v = buf[t] * h;
    }
    buf[t] = v;
  }
  __syncthreads();
  cx<T>* r = fft_pow2(buf, scr, P, nb, tb.tw, -1);
  cx<T>* o = (r == buf) ? scr : buf;
  const cx<T>* kh = (sign < 0) ? tb.khat_f : tb.khat_i;
  for (int t = tid; t < nb * P; t += nth) r[t] = r[t] * kh[t % P];
  __syncthreads();
  r = fft_pow2(r, o, P, nb, tb.tw, +1);
  for (int t = tid; t < nb * P; t += nth) {
    const int k = t % P;
    if (k < N) {
      cx<T> h = tb.chirp[k];
      if (sign > 0) h = conj(h);
      r[t] = r[t] * h;
    }
  }
  __syncthreads();
  return r;
}

// Power-of-two FFT tables of size Q (for the weight correlation of Eq. gmnmp).
template <class T>
struct CorrTab {
  int Q = 0;
  const cx<T>* tw = nullptr;    // [Q] e^{-2 pi i k/Q}
  const cx<T>* what = nullptr;  // [Q] FFT_Q(v)/Q, v[t] = w(-t), t in (-(2L-1), 2L-1) wrapped
};

}  // namespace crv
