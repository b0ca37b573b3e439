// Shared-memory FFT engine for the odd lengths N = 2L_j - 1 of the MW / SO(3)
// grids (Eqs. nodes_alpha..nodes_gamma). A length-N DFT is done by Bluestein's
// chirp-z identity jk = (j^2 + k^2 - (k-j)^2)/2, which turns it into a cyclic
// convolution of length P = 2^p >= 2N-1, done by a register-blocked Stockham
// power-of-two FFT (radix-8 passes, one radix-4 or radix-2 pass when p is not a
// multiple of 3). One code path serves every length (the prime factors of 2L-1
// reach 89 at L = 1024).
//
// A transform is run by a group of P/8 threads (one radix-8 butterfly each per
// pass); several groups share a block and all groups advance in lockstep, so
// block-wide barriers separate the passes. Shared-memory indices are padded by
// one element every 32 to break the bank conflicts of the strided passes.
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
  const cx<T>* hphase = nullptr;  // [N]  e^{+i pi m/N}, m = j (j < (N+1)/2) or j - N: half-sample phase of beta_b
};

// Power-of-two FFT tables of size Q (for the weight correlation of Eq. gmnmp).
template <class T>
struct CorrTab {
  int Q = 0;
  const cx<T>* tw = nullptr;    // [Q] e^{-2 pi i k/Q}
  const cx<T>* what = nullptr;  // [Q] FFT_Q(v)/Q, v[t] = w(-t), t in (-(2L-1), 2L-1) wrapped
};

__host__ __device__ __forceinline__ int padi(int i) { return i + (i >> 5); }
__host__ __device__ __forceinline__ int padded_len(int P) { return P + (P >> 5) + 1; }

template <class T>
__device__ __forceinline__ cx<T> ld_tw(const cx<T>* __restrict__ tw, int idx, int dir) {
  cx<T> w = tw[idx];
  return dir > 0 ? conj(w) : w;
}

// In-register 8-point DFT (decimation in frequency), natural-order output.
template <class T>
__device__ __forceinline__ void dft8(cx<T>* v, int dir) {
  const T s = (T)0.70710678118654752440;
  cx<T> a0 = v[0] + v[4], b0 = v[0] - v[4];
  cx<T> a1 = v[1] + v[5], b1 = v[1] - v[5];
  cx<T> a2 = v[2] + v[6], b2 = v[2] - v[6];
  cx<T> a3 = v[3] + v[7], b3 = v[3] - v[7];
  if (dir < 0) {
    b1 = mk((b1.re + b1.im) * s, (b1.im - b1.re) * s);   // * e^{-i pi/4}
    b2 = mk(b2.im, -b2.re);                              // * -i
    b3 = mk((b3.im - b3.re) * s, -(b3.re + b3.im) * s);  // * e^{-3i pi/4}
  } else {
    b1 = mk((b1.re - b1.im) * s, (b1.re + b1.im) * s);
    b2 = mk(-b2.im, b2.re);
    b3 = mk(-(b3.re + b3.im) * s, (b3.re - b3.im) * s);
  }
  cx<T> c0 = a0 + a2, c2 = a0 - a2, c1 = a1 + a3, d = a1 - a3;
  cx<T> c3 = dir < 0 ? mk(d.im, -d.re) : mk(-d.im, d.re);
  cx<T> e0 = b0 + b2, e2 = b0 - b2, e1 = b1 + b3, f = b1 - b3;
  cx<T> e3 = dir < 0 ? mk(f.im, -f.re) : mk(-f.im, f.re);
  v[0] = c0 + c1; v[4] = c0 - c1; v[2] = c2 + c3; v[6] = c2 - c3;
  v[1] = e0 + e1; v[5] = e0 - e1; v[3] = e2 + e3; v[7] = e2 - e3;
}

// Power-of-two Stockham FFT of one length-P sequence held in x (padded indices), in
// place, run by the Tt = P/8 threads of a group (lane tt). P >= 8. All groups of
// the block must call this together (block barriers between passes).
// dir = -1: X_k = sum x_j e^{-2 pi i jk/P}; dir = +1: e^{+...} (no 1/P).
template <class T>
__device__ void fft_p2(cx<T>* x, int P, const cx<T>* __restrict__ tw, int dir, int tt) {
  const int Q8 = P >> 3;
  int Ns = 1;
  while (Ns < P) {
    const int R = P / Ns;
    if (R >= 8) {
      const int j = tt, k = j & (Ns - 1);
      cx<T> v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = x[padi(j + r * Q8)];
      if (Ns > 1) {
        const int st = P / (8 * Ns);
        const cx<T> w1 = ld_tw(tw, k * st, dir), w2 = w1 * w1, w4 = w2 * w2;
        const cx<T> w3 = w1 * w2, w5 = w1 * w4, w6 = w2 * w4, w7 = w3 * w4;
        v[1] = v[1] * w1; v[2] = v[2] * w2; v[3] = v[3] * w3; v[4] = v[4] * w4;
        v[5] = v[5] * w5; v[6] = v[6] * w6; v[7] = v[7] * w7;
      }
      dft8(v, dir);
      __syncthreads();
      const int out = (j - k) * 8 + k;
#pragma unroll
      for (int r = 0; r < 8; ++r) x[padi(out + r * Ns)] = v[r];
      __syncthreads();
      Ns *= 8;
    } else if (R == 4) {
      cx<T> v[2][4];
      const int Q4 = P >> 2;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = tt + h * Q8, k = j & (Ns - 1);
#pragma unroll
        for (int r = 0; r < 4; ++r) v[h][r] = x[padi(j + r * Q4)];
        if (Ns > 1) {
          const int st = P / (4 * Ns);
          const cx<T> w1 = ld_tw(tw, k * st, dir), w2 = ld_tw(tw, 2 * k * st, dir), w3 = ld_tw(tw, 3 * k * st, dir);
          v[h][1] = v[h][1] * w1; v[h][2] = v[h][2] * w2; v[h][3] = v[h][3] * w3;
        }
        cx<T> a0 = v[h][0] + v[h][2], a1 = v[h][0] - v[h][2], a2 = v[h][1] + v[h][3], d = v[h][1] - v[h][3];
        cx<T> a3 = dir < 0 ? mk(d.im, -d.re) : mk(-d.im, d.re);
        v[h][0] = a0 + a2; v[h][1] = a1 + a3; v[h][2] = a0 - a2; v[h][3] = a1 - a3;
      }
      __syncthreads();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = tt + h * Q8, k = j & (Ns - 1), out = (j - k) * 4 + k;
#pragma unroll
        for (int r = 0; r < 4; ++r) x[padi(out + r * Ns)] = v[h][r];
      }
      __syncthreads();
      Ns *= 4;
    } else {  // R == 2
      cx<T> v[4][2];
      const int Q2 = P >> 1;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int j = tt + h * Q8, k = j & (Ns - 1);
        v[h][0] = x[padi(j)];
        v[h][1] = x[padi(j + Q2)];
        if (Ns > 1) v[h][1] = v[h][1] * ld_tw(tw, k * (P / (2 * Ns)), dir);
        cx<T> a = v[h][0] + v[h][1], b = v[h][0] - v[h][1];
        v[h][0] = a; v[h][1] = b;
      }
      __syncthreads();
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int j = tt + h * Q8, k = j & (Ns - 1), out = (j - k) * 2 + k;
        x[padi(out)] = v[h][0];
        x[padi(out + Ns)] = v[h][1];
      }
      __syncthreads();
      Ns *= 2;
    }
  }
}

// Bluestein core on one sequence: on entry x[padi(j)] holds x_j h^sign_j for j < N
// and 0 for N <= j < P; on exit x[padi(k)] holds the cyclic convolution with the
// chirp kernel, so X_k = h^sign_k * x[padi(k)], k < N. Group-cooperative.
template <class T>
__device__ void bluestein_conv(cx<T>* x, const DftTab<T>& tb, int sign, int tt) {
  const int P = tb.P, Tt = P >> 3;
  fft_p2(x, P, tb.tw, -1, tt);
  const cx<T>* kh = (sign < 0) ? tb.khat_f : tb.khat_i;
  for (int i = tt; i < P; i += Tt) x[padi(i)] = x[padi(i)] * kh[i];
  __syncthreads();
  fft_p2(x, P, tb.tw, +1, tt);
}

template <class T>
__device__ __forceinline__ cx<T> chirp_of(const DftTab<T>& tb, int j, int sign) {
  cx<T> h = tb.chirp[j];
  return sign > 0 ? conj(h) : h;
}

}  // namespace crv
