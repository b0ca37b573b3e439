// Register/shared-memory FFT engine for the odd lengths N = 2L_j - 1 of the MW and
// SO(3) grids (Eqs. nodes_alpha..nodes_gamma). A length-N DFT is done by Bluestein's
// chirp-z identity jk = (j^2 + k^2 - (k-j)^2)/2, which turns it into a cyclic
// convolution of length P = 2^p >= max(16, 2N-1), done with two power-of-two FFTs.
// One code path serves every length (the prime factors of 2L-1 reach 89 at L = 1024).
//
// Power-of-two FFT: Stockham autosort with 16 values per thread. TP = P/16 threads run
// one transform; thread t holds x[t + q TP], q < 16, on entry AND on exit (natural
// order both ways), so consecutive FFTs, pointwise products and the loads and stores
// around them need no reordering. Stage 0 has radix R0 = 2^(p mod 4) (16 when 4 | p)
// and no twiddles; every later stage has radix 16 and builds its twiddles from four
// table values per thread.
// FP32 complex additions run as paired f32x2 instructions (common.cuh); additions of an
// operand rotated by +-i stay scalar (add_rot, sub_rot), so no component swap is needed.
// Between two stages the values pass once through shared memory. Indices there are
// padded by one element every 16, which leaves the exchanges of the P = 4096 transform
// free of bank conflicts. Two exchange buffers alternate, so one barrier per exchange
// suffices: a buffer is rewritten only after the barrier of the exchange in between.
#pragma once
#include "common.cuh"

namespace crv {

// Device tables of one length N in one precision.
template <class T>
struct DftTab {
  int N = 0, P = 0;
  int R0 = 16, nst = 1;           // radix of stage 0 and number of stages of the P-point FFT
  const cx<T>* stw = nullptr;     // stage twiddles: stage s >= 1 (Ns = R0 16^(s-1) points done)
                                  // holds [e][k] = e^{-2 pi i k 2^e / (16 Ns)}, e < 4, k < Ns,
                                  // stages one after another
  const cx<T>* chirp = nullptr;   // [N]  h_t = e^{-i pi t^2 / N}
  const cx<T>* khat_f = nullptr;  // [P]  FFT_P(conj h wrapped) / P   (forward DFT, sign -1)
  const cx<T>* khat_i = nullptr;  // [P]  FFT_P(h wrapped) / P        (inverse DFT, sign +1)
  const cx<T>* hphase = nullptr;  // [N]  e^{+i pi m/N}, m = j (j < (N+1)/2) or j - N: half-sample phase of beta_b
  const cx<T>* bsyn = nullptr;    // [N]  hphase[j] conj(h_j): the beta synthesis's two input factors in one
  const cx<T>* bquad = nullptr;   // [N]  h_k conj(hphase[k]) / N: the beta quadrature's two output factors in one
};

// Weight spectrum for the correlation of Eq. gmnmp (same P as the DftTab of the length).
// Only the even part w_e of the weights enters (see beta_quad_kernel).
template <class T>
struct CorrTab {
  int Q = 0;
  const cx<T>* what = nullptr;  // [Q] FFT_Q(v)/Q, v[t] = w_e(t) = w_e(-t), |t| < 2L-1, wrapped
};


__host__ __device__ __forceinline__ int padx(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int xlen(int P) { return P + (P >> 4); }
// Dynamic shared memory of an FFT block of NT threads: two exchange buffers of NT*16 values.
template <class T> __host__ __device__ inline size_t fft_smem_bytes(int NT) {
  return 2 * (size_t)xlen(16 * NT) * sizeof(cx<T>);
}

// One transform's exchange buffer: element i at p[padx(i) * s].
template <class T>
struct XBuf {
  cx<T>* p;
  int s;
  __device__ __forceinline__ cx<T>& operator[](int i) const { return p[(size_t)padx(i) * s]; }
};
// The two alternating buffers of one transform: buffer h starts at p + h * off.
// take() hands out the next one.
template <class T>
struct XBuf2 {
  cx<T>* p;
  int s, off, cur;
  __device__ __forceinline__ XBuf<T> take() {
    XBuf<T> b{p + (cur ? off : 0), s};
    cur ^= 1;
    return b;
  }
};

// a + d (DIR i) and a - d (DIR i) as scalar operations: a rotated operand would need its
// components swapped to take part in a paired (f32x2) addition.
template <int DIR, class T> __device__ __forceinline__ cx<T> add_rot(cx<T> a, cx<T> d) {
  return DIR < 0 ? mk(a.re + d.im, a.im - d.re) : mk(a.re - d.im, a.im + d.re);
}
template <int DIR, class T> __device__ __forceinline__ cx<T> sub_rot(cx<T> a, cx<T> d) {
  return DIR < 0 ? mk(a.re - d.im, a.im + d.re) : mk(a.re + d.im, a.im - d.re);
}
template <int DIR, class T> __device__ __forceinline__ cx<T> cmulc(cx<T> a, T c, T s) {  // a * (c + DIR i s)
  const T ss = DIR < 0 ? -s : s;
  return mk(a.re * c - a.im * ss, a.re * ss + a.im * c);
}

// 4-point DFT in place, natural order, w = e^{DIR 2 pi i/4}; inputs NZ..3 are zero.
// R2: the input x2 arrives unrotated and is taken as x2 (DIR i).
template <int DIR, int NZ, class T, bool R2 = false>
__device__ __forceinline__ void dft4(cx<T>& x0, cx<T>& x1, cx<T>& x2, cx<T>& x3) {
  if constexpr (NZ == 1) {
    x1 = x0; x2 = x0; x3 = x0;
  } else {
    cx<T> s0, d0, s1, d1;
    if constexpr (NZ == 2) { s0 = x0; d0 = x0; s1 = x1; d1 = x1; }
    else {
      if constexpr (R2) { s0 = add_rot<DIR>(x0, x2); d0 = sub_rot<DIR>(x0, x2); }
      else { s0 = x0 + x2; d0 = x0 - x2; }
      s1 = x1 + x3; d1 = x1 - x3;
    }
    x0 = s0 + s1; x2 = s0 - s1; x1 = add_rot<DIR>(d0, d1); x3 = sub_rot<DIR>(d0, d1);
  }
}

// 8-point DFT (one radix-2 split, then two 4-point DFTs); inputs NZ..7 are zero.
template <int DIR, int NZ, class T>
__device__ __forceinline__ void dft8(cx<T> (&x)[8]) {
  const T c = (T)0.70710678118654752440;
  cx<T> a[4], b[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if constexpr (NZ == 8) { a[r] = x[r] + x[r + 4]; b[r] = x[r] - x[r + 4]; }
    else { a[r] = x[r]; b[r] = x[r]; }
  }
  b[1] = cmulc<DIR>(b[1], c, c);
  // b[2] (twiddle DIR i) is rotated inside the second 4-point DFT
  b[3] = cmulc<DIR>(b[3], -c, c);
  dft4<DIR, 4>(a[0], a[1], a[2], a[3]);
  dft4<DIR, 4, T, true>(b[0], b[1], b[2], b[3]);
#pragma unroll
  for (int k = 0; k < 4; ++k) { x[2 * k] = a[k]; x[2 * k + 1] = b[k]; }
}

// 16-point DFT as 4 x 4: X[k1 + 4 k2] = sum_n2 w16^{n2 k1} w4^{n2 k2} sum_n1 x[4 n1 + n2] w4^{n1 k1}.
// Inputs NZ..15 are zero (NZ = 16 or 8).
template <int DIR, int NZ, class T>
__device__ __forceinline__ void dft16(cx<T> (&x)[16]) {
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173, c2 = (T)0.70710678118654752440;
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<DIR, NZ / 4>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
  // y[n2][k1] sits at x[n2 + 4 k1]; twiddle w16^{n2 k1}
  x[5] = cmulc<DIR>(x[5], c1, s1);      // 1
  x[9] = cmulc<DIR>(x[9], c2, c2);      // 2
  x[13] = cmulc<DIR>(x[13], s1, c1);    // 3
  x[6] = cmulc<DIR>(x[6], c2, c2);      // 2
  // x[10] (twiddle w16^4 = DIR i) is rotated inside the row-2 4-point DFT below
  x[14] = cmulc<DIR>(x[14], -c2, c2);   // 6
  x[7] = cmulc<DIR>(x[7], s1, c1);      // 3
  x[11] = cmulc<DIR>(x[11], -c2, c2);   // 6
  x[15] = cmulc<DIR>(x[15], -c1, -s1);  // 9
  dft4<DIR, 4>(x[0], x[1], x[2], x[3]);
  dft4<DIR, 4>(x[4], x[5], x[6], x[7]);
  dft4<DIR, 4, T, true>(x[8], x[9], x[10], x[11]);
  dft4<DIR, 4>(x[12], x[13], x[14], x[15]);
  // X[k1 + 4 k2] sits at x[4 k1 + k2]
  cx<T> y[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) y[i] = x[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = y[4 * k1 + k2];
}

// Stage 0: B = 16/R butterflies of radix R on v[i + r B], i < B. HIN: v[8..15] are zero.
template <int DIR, int R, bool HIN, class T>
__device__ __forceinline__ void stage0(cx<T> (&v)[16]) {
  constexpr int B = 16 / R;
  if constexpr (R == 16) {
    dft16<DIR, HIN ? 8 : 16>(v);
  } else if constexpr (R == 8) {
#pragma unroll
    for (int i = 0; i < B; ++i) {
      cx<T> a[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) a[r] = v[i + r * B];
      dft8<DIR, HIN ? 4 : 8>(a);
#pragma unroll
      for (int r = 0; r < 8; ++r) v[i + r * B] = a[r];
    }
  } else if constexpr (R == 4) {
#pragma unroll
    for (int i = 0; i < B; ++i) dft4<DIR, HIN ? 2 : 4>(v[i], v[i + B], v[i + 2 * B], v[i + 3 * B]);
  } else {
#pragma unroll
    for (int i = 0; i < B; ++i) {
      if constexpr (HIN) {
        v[i + B] = v[i];
      } else {
        const cx<T> a = v[i] + v[i + B], b = v[i] - v[i + B];
        v[i] = a; v[i + B] = b;
      }
    }
  }
}

// Exchange after a stage of radix R with Ns points done: output r of butterfly
// j = t + i TP goes to (j - k) R + k + r Ns, k = j mod Ns; then thread t reads back
// x[t + q TP]. One barrier between the writes and the reads (buffers alternate).
template <int R, class T>
__device__ __forceinline__ void exchange(cx<T> (&v)[16], XBuf<T> buf, int t, int TP, int Ns) {
  constexpr int B = 16 / R;
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const int j = t + i * TP, k = j & (Ns - 1), base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[base + r * Ns] = v[i + r * B];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = buf[t + q * TP];
}

// Twiddles w^r, r < 16, of one radix-16 butterfly from the table values w, w^2, w^4,
// w^8 (each r is a product of at most 4 of them: at most 3 roundings).
template <class T>
__device__ __forceinline__ void twiddles16(cx<T> w1, cx<T> w2, cx<T> w4, cx<T> w8, cx<T> (&w)[16]) {
  w[1] = w1; w[2] = w2; w[4] = w4; w[8] = w8;
  w[3] = w1 * w2; w[5] = w1 * w4; w[6] = w2 * w4; w[12] = w4 * w8;
  w[7] = w[3] * w4; w[9] = w1 * w8; w[10] = w2 * w8; w[11] = w[3] * w8;
  w[13] = w[5] * w8; w[14] = w[6] * w8; w[15] = w[7] * w8;
}

// Stage structure of a P-point FFT (P = 2^p >= 16): radix of stage 0 and number of stages.
__host__ __device__ constexpr int fft_log2(int P) { return P <= 1 ? 0 : 1 + fft_log2(P >> 1); }
__host__ __device__ constexpr int fft_r0(int P) { return (fft_log2(P) % 4) ? (1 << (fft_log2(P) % 4)) : 16; }
__host__ __device__ constexpr int fft_nst(int P) {
  return 1 + (fft_log2(P) - (fft_r0(P) == 16 ? 4 : fft_log2(P) % 4)) / 4;
}

template <int DIR, bool HIN, class T>
__device__ __forceinline__ void stage0_rt(cx<T> (&v)[16], int R0) {
  switch (R0) {
    case 16: stage0<DIR, 16, HIN>(v); break;
    case 8: stage0<DIR, 8, HIN>(v); break;
    case 4: stage0<DIR, 4, HIN>(v); break;
    default: stage0<DIR, 2, HIN>(v); break;
  }
}
template <class T>
__device__ __forceinline__ void exchange0_rt(cx<T> (&v)[16], XBuf<T> x, int t, int TP, int R0) {
  switch (R0) {
    case 16: exchange<16>(v, x, t, TP, 1); break;
    case 8: exchange<8>(v, x, t, TP, 1); break;
    case 4: exchange<4>(v, x, t, TP, 1); break;
    default: exchange<2>(v, x, t, TP, 1); break;
  }
}

// In-register P-point FFT (no 1/P), w = e^{DIR 2 pi i/P}: v[q] = x[t + q TP] in and out.
// All threads of the block call it together. HIN: x[j] = 0 for j >= P/2 (v[8..15] are
// ignored). PT = P as a compile-time constant (the stage loop unrolls and every index
// folds), or 0 to take P from the table.
template <int DIR, bool HIN, int PT, class T>
__device__ __forceinline__ void fft16(cx<T> (&v)[16], const DftTab<T>& tb, XBuf2<T>& buf, int t) {
  const int P = PT ? PT : tb.P;
  const int TP = P >> 4;
  const int R0 = PT ? fft_r0(PT) : tb.R0;
  const int nst = PT ? fft_nst(PT) : tb.nst;
  if constexpr (PT != 0) stage0<DIR, fft_r0(PT), HIN>(v);
  else stage0_rt<DIR, HIN>(v, R0);
  if (nst == 1) return;
  int Ns = R0;
  const cx<T>* __restrict__ tw = tb.stw;
  // base twiddles of stage 1, fetched before the barrier of the exchange
  int k = t & (Ns - 1);
  cx<T> b1 = tw[k], b2 = tw[Ns + k], b4 = tw[2 * Ns + k], b8 = tw[3 * Ns + k];
  if constexpr (PT != 0) exchange<fft_r0(PT)>(v, buf.take(), t, TP, 1);
  else exchange0_rt(v, buf.take(), t, TP, R0);
  // radix-16 stage s: twiddles from the prefetched base values, butterfly, and (not
  // after the last stage) the next base values and the exchange
  auto stage = [&](int s) {
    cx<T> w[16];
    if (DIR > 0) { b1 = conj(b1); b2 = conj(b2); b4 = conj(b4); b8 = conj(b8); }
    twiddles16(b1, b2, b4, b8, w);
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = v[r] * w[r];
    dft16<DIR, 16>(v);
    if (s + 1 < nst) {
      tw += 4 * Ns;
      const int Nn = Ns * 16;
      k = t & (Nn - 1);
      b1 = tw[k]; b2 = tw[Nn + k]; b4 = tw[2 * Nn + k]; b8 = tw[3 * Nn + k];
      exchange<16>(v, buf.take(), t, TP, Ns);
    }
    Ns *= 16;
  };
  if constexpr (PT != 0) {
#pragma unroll
    for (int s = 1; s < fft_nst(PT); ++s) stage(s);
  } else {
#pragma unroll 1
    for (int s = 1; s < nst; ++s) stage(s);
  }
}

template <class T>
__device__ __forceinline__ cx<T> chirp_of(const DftTab<T>& tb, int j, int sign) {
  cx<T> h = tb.chirp[j];
  return sign > 0 ? conj(h) : h;
}

}  // namespace crv
