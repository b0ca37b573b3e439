// Kernels of the spin SHT and the Wigner transforms (Sec. III-A-2), templated on
// the working precision T (double for the plain path, float for the mixed path).
//
// Index sets of one transform of band limit Lb (N = 2Lb-1):
//   m = m0 + mi, mi < Mc      (m0 = 0, Mc = Lb for real signals; m0 = -(Lb-1), Mc = N otherwise)
//   n = n0 + nstep * ni, ni < Nc   (spin 0: even n only, nstep = 2; else nstep = 1; the
//                                   kernels rely on nstep being 1 or 2)
//   m' = 0..Lb-1              (X_{m n, -m'} = (-1)^{m+n} X_{m n m'}, so only m' >= 0 is kept)
// Volumes are stored [row][mi][ni] with ni fastest.
#pragma once
#include <type_traits>
#include <utility>

#include "fft.cuh"

namespace crv {

struct ColSet {
  int Mc, m0, Nc, n0, nstep;
  int extra;    // added to m+n in parities and phases (spin for the SHT)
  FastDiv fNc;  // division by Nc
  // Column of (mi, ni) in an (m, n) plane: the columns (2i, ni) and (2i + 1, ni) (m and m + 1
  // at one n, the pairs of the beta transforms) are adjacent, so consecutive pairs fill whole
  // sectors: c = ((mi / 2) Nc + ni) 2 + mi % 2. A plane holds pitch() columns (one unused
  // column per n when Mc is odd); with Nc = 1 (the SHT) c = mi.
  __host__ __device__ __forceinline__ int col(int mi, int ni) const { return (((mi >> 1) * Nc + ni) << 1) | (mi & 1); }
  __host__ __device__ __forceinline__ size_t pitch() const { return (size_t)((Mc + 1) >> 1) * Nc * 2; }
};

// L1 prefetch of a global address (no register results): loaders that define
// pf(c, j) have the inputs of their next sequence fetched while the current one runs
// (measured: faster for the ring rows, neutral for ring columns, and much slower for the
// beta columns read from HBM at a stride of a whole (m, n) plane, which do without).
__device__ __forceinline__ void pf_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
template <class Ld, class = void> struct HasPf { static constexpr bool value = false; };
template <class Ld>
struct HasPf<Ld, decltype(std::declval<const Ld&>().pf(0, 0), void())> { static constexpr bool value = true; };

// ---------------------------------------------------------------------------
// Batched DFTs of length N (Bluestein on the register FFT of fft.cuh). A block of
// NT threads runs G = NT / TP transforms at a time, TP = P/16 threads each.
//
// COLS = false (rows): sequence c is gathered by ld(c, j), j < N, typically a
//   contiguous row; a transform's threads are consecutive, so loads run along j.
// COLS = true (columns): consecutive sequences are adjacent in memory; the G
//   transforms of a block interleave their threads (g fastest), so each load or
//   store touches G adjacent sequences, and the exchange buffers interleave too.
// Storers get st(c, k, X_k, X_k') for every k < N, where k' is set by Mirror<St>:
// 0: no partner (X_k' = X_k), 1: k' = (N - k) mod N (real-pair unpacking), 2: k' = N - 1 - k;
// the partner is gathered through shared memory.
// ---------------------------------------------------------------------------
template <class St> struct Mirror { static constexpr int value = 0; };

template <class T, int NT, bool COLS, int PT>
__device__ __forceinline__ void fft_slot(int& g, int& t, XBuf2<T>& buf, unsigned char* smraw, int Prt) {
  const int P = PT ? PT : Prt;
  const int TP = P >> 4, G = NT / TP, XL = xlen(P);
  cx<T>* sm = reinterpret_cast<cx<T>*>(smraw);
  if (COLS) { g = threadIdx.x % G; t = threadIdx.x / G; }
  else { g = threadIdx.x / TP; t = threadIdx.x % TP; }
  buf.p = COLS ? sm + g : sm + (size_t)g * XL;
  buf.s = COLS ? G : 1;
  buf.off = G * XL;
  buf.cur = 0;
}

// The FP32 beta transforms stage the spectra they multiply by (Bluestein's kernel, the weight
// spectrum of the quadrature) in shared memory after the exchange buffers, once per block: every
// column pair then reads them there instead of through L1 (and the quadrature no longer spills
// registers). FP64 blocks have no room left for them.
template <class T> __host__ __device__ constexpr bool kStageSpectra() { return sizeof(T) == 4; }
template <class T> __host__ __device__ inline size_t fft_smem_bytes_tabs(int NT, int P, int ntab) {
  return fft_smem_bytes<T>(NT) + (kStageSpectra<T>() ? (size_t)ntab * P * sizeof(cx<T>) : 0);
}
// Copy n tables of P values into the staging area (all threads of the block; ends with a
// barrier) and return its start; without staging return nullptr.
template <class T, int NT>
__device__ __forceinline__ const cx<T>* stage_spectra(unsigned char* smraw, int P, const cx<T>* a,
                                                      const cx<T>* b = nullptr) {
  if constexpr (!kStageSpectra<T>()) {
    return nullptr;
  } else {
    cx<T>* s = reinterpret_cast<cx<T>*>(smraw + fft_smem_bytes<T>(NT));
    for (int i = threadIdx.x; i < P; i += NT) {
      s[i] = a[i];
      if (b) s[P + i] = b[i];
    }
    __syncthreads();
    return s;
  }
}

// Blocks of NT threads; FP32 blocks of 256 threads fit twice on an SM (<= 128 registers).
template <class T, int NT> struct FftMinBlocks { static constexpr int value = (sizeof(T) == 4 && NT <= 256) ? 2 : 1; };

// PT: P as a compile-time constant, or 0 (from the table). Blocks stride through the
// sequences together, so that neighbouring blocks fill each sector of a large output at
// about the same time (measured faster than contiguous runs per block here).
template <class T, int NT, bool COLS, int PT, class Ld, class St>
__global__ void __launch_bounds__(NT, (FftMinBlocks<T, NT>::value)) dft_kernel(DftTab<T> tb, int sign, int nseq, Ld ld, St st) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = tb.N, TP = (PT ? PT : tb.P) >> 4, G = NT / TP;
  int g, t;
  XBuf2<T> buf;
  fft_slot<T, NT, COLS, PT>(g, t, buf, smraw, tb.P);
  // the kernel spectrum is read through L1 here: the ring transforms' strided loads need the L1
  // that staging it in shared memory would take (measured: staging it made them 4-15 % slower)
  const cx<T>* __restrict__ kh = (sign < 0) ? tb.khat_f : tb.khat_i;
  const int s_end = nseq, s_step = gridDim.x * G;
  for (int s0 = blockIdx.x * G; s0 < s_end; s0 += s_step) {
    const int c = s0 + g;
    const bool valid = c < nseq;
    cx<T> v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {  // j < N <= P/2 only for q < 8
      const int j = t + q * TP;
      v[q] = mk<T>(0, 0);
      if (q < 8 && valid && j < N) v[q] = ld(c, j) * chirp_of(tb, j, sign);
    }
    if constexpr (HasPf<Ld>::value) {
      const int cn = c + s_step;
      if (cn < s_end) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = t + q * TP;
          if (j < N) ld.pf(cn, j);
        }
      }
    }
    fft16<-1, true, PT>(v, tb, buf, t);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = v[q] * kh[t + q * TP];
    fft16<+1, false, PT>(v, tb, buf, t);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = t + q * TP;
      v[q] = v[q] * chirp_of(tb, k < N ? k : 0, sign);
    }
    if constexpr (Mirror<St>::value != 0) {
      const XBuf<T> x = buf.take();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = t + q * TP;
        if (k < N) x[k] = v[q];
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = t + q * TP;
        const int kp = Mirror<St>::value == 1 ? (k == 0 ? 0 : N - k) : N - 1 - k;
        if (valid && k < N) st(c, k, v[q], x[kp]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = t + q * TP;
        if (valid && k < N) st(c, k, v[q], v[q]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Loaders / storers
// ---------------------------------------------------------------------------

// Column pairs. Columns c_A = (2 i, ni) and c_B = (2 i + 1, ni) (m and m + 1, one n) have
// opposite parities of m + n + extra, so one of their beta extensions is symmetric under
// b -> N-1-b (m' -> -m') and the other antisymmetric: one DFT of the sum serves both and
// the halves separate by that reflection. Pair index p = i * Nc + ni; c_B = -1 if 2i+1 = Mc.
struct ColPair {
  int cA, cB, parA;  // parA = parity of m + n + extra of column A (B has the other)
  int mA, n;         // m of column A (B: mA + 1) and n of both
};
__device__ __forceinline__ ColPair col_pair(const ColSet& cs, int p) {
  const int i = (int)cs.fNc.div((uint32_t)p), ni = p - i * cs.Nc;
  ColPair r;
  r.cA = cs.col(2 * i, ni);
  r.cB = (2 * i + 1 < cs.Mc) ? r.cA + 1 : -1;
  r.mA = cs.m0 + 2 * i;
  r.n = cs.n0 + cs.nstep * ni;
  r.parA = (r.mA + r.n + cs.extra) & 1;
  return r;
}
__host__ __device__ inline int num_col_pairs(const ColSet& cs) { return (cs.Mc + 1) / 2 * cs.Nc; }
// Optional list of the column pairs a beta transform visits (the others are known to be
// zero and are neither read nor written): pair idx[q], q < n; idx = nullptr visits all.
struct PairMap {
  const int* idx = nullptr;
  int n = 0;
};


// Ring inverse, step over n: sequence (b, mi) of the planes Xb[b] -> T[b][mi][g].
// Z (unrotated curvelets): columns |n| < nlo and |m| > |n| are zero and are not read.
template <class T, bool Z = false>
struct LdRingN {
  const cx<T>* Xb; ColSet cs; int N; FastDiv fMc;
  int nlo = 0;
  __device__ cx<T> operator()(int c, int j) const {
    const int b = (int)fMc.div((uint32_t)c), mi = c - b * cs.Mc;
    // j = n mod N; find ni with n0 + nstep*ni == n
    int n = (j <= (N - 1) / 2) ? j : j - N;
    int d = n - cs.n0;
    if (d < 0 || (d & (cs.nstep - 1))) return mk<T>(0, 0);
    const int ni = d >> (cs.nstep - 1);
    if (ni >= cs.Nc) return mk<T>(0, 0);
    if constexpr (Z) {
      const int an = n < 0 ? -n : n, m = cs.m0 + mi;
      if (an < nlo || (m < 0 ? -m : m) > an) return mk<T>(0, 0);
    }
    return Xb[(size_t)b * cs.pitch() + cs.col(mi, ni)];
  }
};
template <class T>
struct StContig {  // out[c][k], k < N, rows of S elements
  cx<T>* out; int S;
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const { out[(size_t)c * S + k] = v; }
};

// Ring inverse, step over m: column (b, g) of T[b][mi][g] -> W[b][a][g].
// real: Hermitian completion z_{N-m} = conj(z_m), output real part.
template <class T>
struct LdRingM {  // T[b][mi][g], rows of S >= N elements
  const cx<T>* Tb; int Mc, m0, N, S; bool real; FastDiv fN;
  __device__ cx<T> operator()(int c, int j) const {
    const int b = (int)fN.div(c), g = c - b * N;
    const cx<T>* base = Tb + (size_t)b * Mc * S + g;
    int m = (j <= (N - 1) / 2) ? j : j - N;
    if (real) {
      if (m >= 0) return base[(size_t)m * S];
      return conj(base[(size_t)(-m) * S]);
    }
    int mi = m - m0;
    if (mi < 0 || mi >= Mc) return mk<T>(0, 0);
    return base[(size_t)mi * S];
  }
};
template <class T, class OutT>
struct StW {  // W[b][a][g] in OutT, real or complex
  OutT* W; int N; bool real; FastDiv fN;
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const {
    const int b = (int)fN.div(c), g = c - b * N;
    const size_t idx = ((size_t)b * N + k) * N + g;
    if (real) W[idx] = (OutT)v.re;
    else { W[2 * idx] = (OutT)v.re; W[2 * idx + 1] = (OutT)v.im; }
  }
};

// Ring forward, step over g: row (b, a) of W -> U[b][a][ni] (scaled 1/N).
template <class T, class InT>
struct LdWRow {
  const InT* W; int N; bool real;
  __device__ cx<T> operator()(int c, int j) const {
    const size_t idx = (size_t)c * N + j;
    if (real) return mk<T>((T)W[idx], (T)0);
    return mk<T>((T)W[2 * idx], (T)W[2 * idx + 1]);
  }
};
template <class T>
struct StRingN {  // U[c][ni] = D[n mod N] / N for n in the n-set
  cx<T>* U; int Nc, n0, nstep, N; T scale;
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const {
    int n = (k <= (N - 1) / 2) ? k : k - N;
    int d = n - n0;
    if (d < 0 || (d & (nstep - 1))) return;
    const int ni = d >> (nstep - 1);
    if (ni < Nc) U[(size_t)c * Nc + ni] = v * scale;
  }
};
// Ring forward, step over a: column (b, ni) of U[b][a][ni] -> Xb[b][mi][ni].
template <class T>
struct LdRingA {
  const cx<T>* U; int Nc, N; FastDiv fNc;
  __device__ cx<T> operator()(int c, int j) const {
    const int b = (int)fNc.div(c), ni = c - b * Nc;
    return U[((size_t)b * N + j) * Nc + ni];
  }
};
template <class T>
struct StRingA {
  cx<T>* Xb; ColSet cs; int N; T scale;
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const {
    const int b = (int)cs.fNc.div((uint32_t)c), ni = c - b * cs.Nc;
    int m = (k <= (N - 1) / 2) ? k : k - N;
    int mi = m - cs.m0;
    if (mi >= 0 && mi < cs.Mc) Xb[(size_t)b * cs.pitch() + cs.col(mi, ni)] = v * scale;
  }
};

// Real pairs. Forward over g for real W: rows 2c and 2c+1 of the chunk packed as
// x + i y; X_k = (Z_k + conj Z_{-k})/2, Y_k = (Z_k - conj Z_{-k})/(2i).
template <class T, class InT>
struct LdWRowPair {
  const InT* W; int N, nrows;
  __device__ cx<T> operator()(int c, int j) const {
    const int r0 = 2 * c, r1 = 2 * c + 1;
    const T x = (T)W[(size_t)r0 * N + j];
    const T y = (r1 < nrows) ? (T)W[(size_t)r1 * N + j] : (T)0;
    return mk<T>(x, y);
  }
  __device__ void pf(int c, int j) const {
    pf_l1(W + (size_t)(2 * c) * N + j);
    if (2 * c + 1 < nrows) pf_l1(W + (size_t)(2 * c + 1) * N + j);
  }
};
template <class T>
struct StRingNPair {
  cx<T>* U; int Nc, n0, nstep, N, nrows; T scale;
  __device__ void operator()(int c, int k, cx<T> z, cx<T> zn) const {
    int n = (k <= (N - 1) / 2) ? k : k - N;
    int d = n - n0;
    if (d < 0 || (d & (nstep - 1))) return;
    const int ni = d >> (nstep - 1);
    if (ni >= Nc) return;
    const T h = scale * (T)0.5;
    const cx<T> a = mk<T>((z.re + zn.re) * h, (z.im - zn.im) * h);   // (z + conj zn)/2
    const cx<T> b = mk<T>((z.im + zn.im) * h, (zn.re - z.re) * h);   // (z - conj zn)/(2i)
    U[(size_t)(2 * c) * Nc + ni] = a;
    if (2 * c + 1 < nrows) U[(size_t)(2 * c + 1) * Nc + ni] = b;
  }
};
template <class T> struct Mirror<StRingNPair<T>> { static constexpr int value = 1; };
// ---------------------------------------------------------------------------
// Ring transforms of real signals. Only m >= 0 is kept (all n), and F_{-m,-n} =
// conj F_{m,n}, so each direction needs the columns n >= 0 only: h = n / nstep < Nh,
// column ni = ni0 + h of the n-set, whose mirror column Nc - 1 - ni holds -n (the n-set
// is symmetric). Ring buffers are laid out [b][a][h].
// ---------------------------------------------------------------------------
// Analysis, step over m (sign +1) for n >= 0: column (b, h) of Xb[b][mi][ni], extended to
// m < 0 by the conjugate of the -n column -> R[b][a][h].
// Z (unrotated curvelets): the columns start at h0, and entries |m| > n are zero and not read.
template <class T, bool Z = false>
struct LdRingMHalf {
  const cx<T>* Xb; ColSet cs; int ni0, N, Nh; FastDiv fNh;  // Nh columns per ring, from h0 on
  int h0 = 0;
  __device__ const cx<T>* at(int c, int j, int& m, bool& z) const {
    const int b = (int)fNh.div((uint32_t)c), h = (Z ? h0 : 0) + (c - b * Nh), ni = ni0 + h;
    m = (j <= (N - 1) / 2) ? j : j - N;
    z = Z && (m < 0 ? -m : m) > h * cs.nstep;
    const cx<T>* base = Xb + (size_t)b * cs.pitch();
    return m >= 0 ? base + cs.col(m, ni) : base + cs.col(-m, cs.Nc - 1 - ni);
  }
  __device__ cx<T> operator()(int c, int j) const {
    int m;
    bool z;
    const cx<T>* q = at(c, j, m, z);
    if (z) return mk<T>(0, 0);
    const cx<T> v = *q;
    return m >= 0 ? v : conj(v);
  }
  __device__ void pf(int c, int j) const {
    int m;
    bool z;
    const cx<T>* q = at(c, j, m, z);
    if (!z) pf_l1(q);
  }
};
template <class T>
struct StRingMHalf {  // R[b][a][h0 + h], rows of Rp columns; Nh columns per ring
  cx<T>* R; int N, Nh; FastDiv fNh; int Rp, h0;
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const {
    const int b = (int)fNh.div((uint32_t)c), h = c - b * Nh;
    R[((size_t)b * N + k) * Rp + h0 + h] = v;
  }
};
// Analysis, step over n (sign +1) with real output: rows a1 = 2 ap and a2 = 2 ap + 1 of
// R[b][a][h], each extended Hermitian in n (n < 0: conjugate of -n), packed as x + i y;
// the transform's real and imaginary parts are the two rows of W.
// Z (unrotated curvelets): |n| < nlo is zero (those columns of R are not written).
template <class T, bool Z = false>
struct LdRingNHerm {
  const cx<T>* R; int N, Nh, nstep, npair; FastDiv fP;
  int nlo = 0;
  __device__ cx<T> operator()(int c, int j) const {
    const int b = (int)fP.div((uint32_t)c), a1 = 2 * (c - b * npair), a2 = a1 + 1;
    const int n = (j <= (N - 1) / 2) ? j : j - N;
    const int an = n < 0 ? -n : n;
    if ((an & (nstep - 1)) || (Z && an < nlo)) return mk<T>(0, 0);
    const int h = an >> (nstep - 1);
    const cx<T>* rb = R + (size_t)b * N * Nh;
    cx<T> x = rb[(size_t)a1 * Nh + h];
    cx<T> y = (a2 < N) ? rb[(size_t)a2 * Nh + h] : mk<T>(0, 0);
    if (n < 0) { x = conj(x); y = conj(y); }
    return mk<T>(x.re - y.im, x.im + y.re);
  }
  __device__ void pf(int c, int j) const {
    const int b = (int)fP.div((uint32_t)c), a1 = 2 * (c - b * npair);
    const int n = (j <= (N - 1) / 2) ? j : j - N;
    const int an = n < 0 ? -n : n;
    if ((an & (nstep - 1)) || (Z && an < nlo)) return;
    const cx<T>* q = R + (size_t)b * N * Nh + (size_t)a1 * Nh + (an >> (nstep - 1));
    pf_l1(q);
    if (a1 + 1 < N) pf_l1(q + Nh);
  }
};
template <class T, class OutT>
struct StWRowPair {  // W[b][a][g], real: row a1 <- Re, a2 <- Im
  OutT* W; int N, npair; FastDiv fP;
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const {
    const int b = (int)fP.div((uint32_t)c), a1 = 2 * (c - b * npair), a2 = a1 + 1;
    W[((size_t)b * N + a1) * N + k] = (OutT)v.re;
    if (a2 < N) W[((size_t)b * N + a2) * N + k] = (OutT)v.im;
  }
};
// Synthesis, step over g (sign -1) of real rows in pairs (LdWRowPair), keeping n >= 0:
// U[b][a][h] = D_n / N.
template <class T>
struct StRingNPairHalf {
  cx<T>* U; int Nh, nstep, N, nrows; T scale;
  int h0 = 0;  // columns h < h0 are not needed
  __device__ void operator()(int c, int k, cx<T> z, cx<T> zn) const {
    if (k > (N - 1) / 2 || (k & (nstep - 1))) return;  // n = k >= 0 in the n-set
    const int h = k >> (nstep - 1);
    if (h >= Nh || h < h0) return;
    const T hs = scale * (T)0.5;
    U[(size_t)(2 * c) * Nh + h] = mk<T>((z.re + zn.re) * hs, (z.im - zn.im) * hs);
    if (2 * c + 1 < nrows) U[(size_t)(2 * c + 1) * Nh + h] = mk<T>((z.im + zn.im) * hs, (zn.re - z.re) * hs);
  }
};
template <class T> struct Mirror<StRingNPairHalf<T>> { static constexpr int value = 1; };
// Synthesis, step over a (sign -1) for n >= 0: column (b, h) of U[b][a][h] -> D_m; the
// m >= 0 outputs go to column ni of Xb, and conj(D_{-m}) to the mirror column (-n).
template <class T>
struct LdRingAHalf {  // U[b][a][h0 + h], rows of Up columns; Nh columns per ring
  const cx<T>* U; int N, Nh; FastDiv fNh; int Up, h0;
  __device__ const cx<T>* at(int c, int j) const {
    const int b = (int)fNh.div((uint32_t)c), h = h0 + (c - b * Nh);
    return U + ((size_t)b * N + j) * Up + h;
  }
  __device__ cx<T> operator()(int c, int j) const { return *at(c, j); }
  __device__ void pf(int c, int j) const { pf_l1(at(c, j)); }
};
template <class T>
struct StRingAHalf {
  cx<T>* Xb; ColSet cs; int ni0, N, Nh; T scale; FastDiv fNh;  // Nh columns per ring, from h0 on
  int h0 = 0;
  __device__ void operator()(int c, int k, cx<T> v, cx<T> vn) const {
    if (k >= cs.Mc) return;  // m = k >= 0 (Mc = Lb <= (N + 1) / 2)
    const int b = (int)fNh.div((uint32_t)c), h = h0 + (c - b * Nh), ni = ni0 + h;
    cx<T>* plane = Xb + (size_t)b * cs.pitch();
    plane[cs.col(k, ni)] = v * scale;
    if (h > 0) plane[cs.col(k, cs.Nc - 1 - ni)] = conj(vn) * scale;
  }
};
template <class T> struct Mirror<StRingAHalf<T>> { static constexpr int value = 1; };

// SHT: map ring t -> F[t][mi] (1/N scaled), real or complex double map.
struct LdMapRow {
  const double* map; int N; bool real;
  template <class T> __device__ cx<T> get(int c, int j) const {
    const size_t idx = (size_t)c * N + j;
    if (real) return mk<T>((T)map[idx], (T)0);
    return mk<T>((T)map[2 * idx], (T)map[2 * idx + 1]);
  }
};
template <class T>
struct LdMapRowT {
  LdMapRow r;
  __device__ cx<T> operator()(int c, int j) const { return r.template get<T>(c, j); }
};
template <class T>
struct StSHTRow {  // F[c][mi] for m in m-set
  cx<T>* F; int Mc, m0, N; T scale;
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const {
    int m = (k <= (N - 1) / 2) ? k : k - N;
    int mi = m - m0;
    if (mi >= 0 && mi < Mc) F[(size_t)c * Mc + mi] = v * scale;
  }
};
// SHT inverse phi step: row t of F[t][mi] -> map[t][p]
template <class T>
struct LdSHTRow {
  const cx<T>* F; int Mc, m0, N; bool real;
  __device__ cx<T> operator()(int c, int j) const {
    const cx<T>* base = F + (size_t)c * Mc;
    int m = (j <= (N - 1) / 2) ? j : j - N;
    if (real) return (m >= 0) ? base[m] : conj(base[-m]);
    int mi = m - m0;
    return (mi >= 0 && mi < Mc) ? base[mi] : mk<T>(0, 0);
  }
};
struct StMapRow {
  double* map; int N; bool real;
  template <class T> __device__ void operator()(int c, int k, cx<T> v, cx<T>) const {
    const size_t idx = (size_t)c * N + k;
    if (real) map[idx] = (double)v.re;
    else { map[2 * idx] = (double)v.re; map[2 * idx + 1] = (double)v.im; }
  }
};

// ---------------------------------------------------------------------------
// Extension of a column pair to the 2Lb-1 nodes of the full circle (beta transforms).
// Rows i < Lb of the two columns are loaded once (they sit in v[0..3]: Lb <= P/4), and
// the reflected half, sA (A - B) with sA = (-1)^{parA}, comes back through shared memory:
//   v[q] = (A + B)_j for j < Lb,  sA (A - B)_{N - off - j} for Lb <= j < N, 0 beyond,
// with off = 0 when index 0 is its own mirror (m' -> -m') and off = 1 for the reflection
// b -> N - 1 - b of the ring samples.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void load_pair_ext(cx<T> (&v)[16], const cx<T>* __restrict__ X, int C, const ColPair& cp,
                                              bool valid, int Lb, int N, int t, int TP, int off, XBuf2<T>& buf) {
  cx<T> d[4];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = mk<T>(0, 0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = t + q * TP;
    d[q] = mk<T>(0, 0);
    if (valid && j < Lb) {
      const cx<T>* row = X + (size_t)j * C;
      const cx<T> a = row[cp.cA];
      const cx<T> b = cp.cB >= 0 ? row[cp.cB] : mk<T>(0, 0);
      v[q] = a + b;
      d[q] = cp.parA ? b - a : a - b;
    }
  }
  const XBuf<T> x = buf.take();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = t + q * TP;
    if (j < Lb) x[j] = d[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = t + q * TP;
    if (j >= Lb && j < N) v[q] = x[N - off - j];
  }
}

// ---------------------------------------------------------------------------
// Synthesis over beta of a column pair (Eq. inverse_feul, the m' -> beta step):
// z_{m'} = (X~A + X~B)_{m'} e^{i m' pi/N} on m' in (-Lb, Lb), X~_{-m'} = (-1)^{m+n+extra} X~_{m'};
// F_b = sum_{m'} z_{m'} e^{2 pi i m' b/N}; the symmetric half (F_b + F_{N-1-b})/2 belongs to the
// column of even parity, the antisymmetric half to the other. In: X[m'][c] (m' < Lb);
// out: Y[b][c] (b < Lb). Threads as in dft_kernel with COLS.
// ---------------------------------------------------------------------------
template <class T, int NT, int PT>
__global__ void __launch_bounds__(NT, (FftMinBlocks<T, NT>::value)) beta_synth_kernel(DftTab<T> tb, int ncols, int Lb,
                                                                     const cx<T>* __restrict__ X,
                                                                     cx<T>* __restrict__ Y, ColSet cs, PairMap pm) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = tb.N, TP = (PT ? PT : tb.P) >> 4, G = NT / TP;
  const int npair = pm.idx ? pm.n : num_col_pairs(cs);
  int g, t;
  XBuf2<T> buf;
  fft_slot<T, NT, true, PT>(g, t, buf, smraw, tb.P);
  const cx<T>* khat = tb.khat_i;
  if (const cx<T>* st = stage_spectra<T, NT>(smraw, PT ? PT : tb.P, khat)) khat = st;
  const int span = (npair + gridDim.x * G - 1) / (gridDim.x * G) * G;
  const int s_end = min(npair, (blockIdx.x + 1) * span);
  for (int s0 = blockIdx.x * span; s0 < s_end; s0 += G) {
    const int p = s0 + g;
    const bool valid = p < s_end;
    const ColPair cp = valid ? col_pair(cs, pm.idx ? pm.idx[p] : p) : ColPair{0, -1, 0};
    cx<T> v[16];
    load_pair_ext<T>(v, X, ncols, cp, valid, Lb, N, t, TP, 0, buf);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = t + q * TP;
      if (j < N) v[q] = v[q] * tb.bsyn[j];
    }
    fft16<-1, true, PT>(v, tb, buf, t);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = v[q] * khat[t + q * TP];
    fft16<+1, false, PT>(v, tb, buf, t);
    const XBuf<T> y = buf.take();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = t + q * TP;
      if (k < N) {
        v[q] = v[q] * chirp_of(tb, k, +1);
        y[k] = v[q];
      }
    }
    __syncthreads();
    if (valid) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = t + q * TP;
        if (k < Lb) {
          const cx<T> r = y[N - 1 - k];
          const cx<T> sym = (v[q] + r) * (T)0.5, anti = (v[q] - r) * (T)0.5;
          Y[(size_t)k * ncols + cp.cA] = cp.parA ? anti : sym;
          if (cp.cB >= 0) Y[(size_t)k * ncols + cp.cB] = cp.parA ? sym : anti;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Exact quadrature over beta (Eqs. TildaFmn, Fmnmp, gmnmp), folded onto m' >= 0, for a
// column pair (ColPair): extend the Lb ring values of each column to 2Lb-1 with
// (-1)^{m+n+extra} and add the two, DFT (sign -1, half-sample phase e^{-i m'' pi/N}/N),
// correlate with the even part w_e of the weights (precomputed transform of
// v[t] = w_e(t) on Q = P points), and unfold: with Yt = D * w_e,
//   Yhat_sym(m') = Yt(m') + Yt(-m')  (m' > 0; Yt(0) at m' = 0),
//   Yhat_anti(m') = Yt(m') - Yt(-m') (m' > 0; 0 at m' = 0),
// the symmetric one for the column of even parity; then scale * i^{m pa + n pb + pc}.
// This equals the fold Y(m') + (-1)^{m+n+extra} Y(-m') of the full-weight correlation of
// each column: the odd weights (p = +-1) cancel in that fold, and the even (odd) part of
// the DFT of a symmetric (antisymmetric) extension is all of it.
// In: Xb[b][c] (b < Lb, rows of ncols columns); out: Y[m'][c] (m' < Lb). Threads as in
// dft_kernel with COLS.
// ---------------------------------------------------------------------------
template <class T, int NT, int PT>
__global__ void __launch_bounds__(NT, (FftMinBlocks<T, NT>::value)) beta_quad_kernel(DftTab<T> tb, CorrTab<T> ct, int ncols, int Lb,
                                                                    const cx<T>* __restrict__ Xb,
                                                                    cx<T>* __restrict__ Y, ColSet cs, T scale, int pa,
                                                                    int pb, int pc, PairMap pm) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = tb.N, Q = PT ? PT : ct.Q, TP = (PT ? PT : tb.P) >> 4, G = NT / TP;
  const int npair = pm.idx ? pm.n : num_col_pairs(cs);
  int g, t;
  XBuf2<T> buf;
  fft_slot<T, NT, true, PT>(g, t, buf, smraw, tb.P);
  const cx<T>* khat = tb.khat_f;
  const cx<T>* what = ct.what;
  if (const cx<T>* st = stage_spectra<T, NT>(smraw, PT ? PT : tb.P, khat, what)) {
    khat = st;
    what = st + (PT ? PT : tb.P);
  }
  const int span = (npair + gridDim.x * G - 1) / (gridDim.x * G) * G;
  const int s_end = min(npair, (blockIdx.x + 1) * span);
  for (int s0 = blockIdx.x * span; s0 < s_end; s0 += G) {
    const int p = s0 + g;
    const bool valid = p < s_end;
    cx<T> v[16];
    {
      // extensions to the 2Lb-1 nodes of the full circle, summed, then the chirp (the pair's
      // descriptor is rebuilt for the unfold below rather than kept live across the FFTs)
      const ColPair cp = valid ? col_pair(cs, pm.idx ? pm.idx[p] : p) : ColPair{0, -1, 0};
      load_pair_ext<T>(v, Xb, ncols, cp, valid, Lb, N, t, TP, 1, buf);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = t + q * TP;
      if (j < N) v[q] = v[q] * chirp_of(tb, j, -1);
    }
    fft16<-1, true, PT>(v, tb, buf, t);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = v[q] * khat[t + q * TP];
    fft16<+1, false, PT>(v, tb, buf, t);
    // u_{m''} at index m'' mod Q: D_{m'' mod N} h_k e^{-i m'' pi/N} / N; zero for Lb <= index <= Q - Lb
    {
      const XBuf<T> x = buf.take();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int k = t + q * TP;
        if (q < 8 && k < N) x[k < Lb ? k : k - N + Q] = v[q] * tb.bquad[k];
        if (k >= Lb && k <= Q - Lb) x[k] = mk<T>(0, 0);
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = x[t + q * TP];
    }
    fft16<-1, false, PT>(v, tb, buf, t);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = v[q] * what[t + q * TP];
    fft16<+1, false, PT>(v, tb, buf, t);
    // unfold into the two columns
    const XBuf<T> y = buf.take();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = t + q * TP;
      if (i > Q - Lb) y[i] = v[q];
    }
    __syncthreads();
    if (valid) {
      const ColPair cp = col_pair(cs, pm.idx ? pm.idx[p] : p);
      const int phA = imod(cp.mA * pa + cp.n * pb + pc, 4), phB = imod((cp.mA + 1) * pa + cp.n * pb + pc, 4);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int mp = t + q * TP;
        if (mp < Lb) {
          cx<T> sym = v[q], anti = mk<T>(0, 0);
          if (mp > 0) {
            const cx<T> w = y[Q - mp];
            anti = sym - w;
            sym = sym + w;
          }
          Y[(size_t)mp * ncols + cp.cA] = mul_ipow((cp.parA ? anti : sym) * scale, phA);
          if (cp.cB >= 0) Y[(size_t)mp * ncols + cp.cB] = mul_ipow((cp.parA ? sym : anti) * scale, phB);
        }
      }
    }
  }
}

}  // namespace crv
