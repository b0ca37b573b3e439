// Kernels of the spin SHT and the Wigner transforms (Sec. III-A-2), templated on
// the working precision T (double for the plain path, float for the mixed path).
//
// Index sets of one transform of band limit Lb (N = 2Lb-1):
//   m = m0 + mi, mi < Mc      (m0 = 0, Mc = Lb for real signals; m0 = -(Lb-1), Mc = N otherwise)
//   n = n0 + nstep * ni, ni < Nc   (spin 0: even n only, nstep = 2; else nstep = 1)
//   m' = 0..Lb-1              (X_{m n, -m'} = (-1)^{m+n} X_{m n m'}, so only m' >= 0 is kept)
// Volumes are stored [row][mi][ni] with ni fastest.
#pragma once
#include "fft.cuh"

namespace crv {

struct ColSet {
  int Mc, m0, Nc, n0, nstep;
  int extra;  // added to m+n in parities and phases (spin for the SHT)
  __device__ __forceinline__ int m_of(int c) const { return m0 + c / Nc; }
  __device__ __forceinline__ int n_of(int c) const { return n0 + nstep * (c % Nc); }
};

// ---------------------------------------------------------------------------
// Generic batched DFT over columns: for each column c < ncols, a length-N input
// gathered by ld(c, j), a length-N DFT with the given sign, and st(c, k, value)
// for every output k < N (the storer decides which to keep). COLFAST = true when
// consecutive columns are adjacent in memory (load/store loops then run over
// columns fastest, for coalescing).
// ---------------------------------------------------------------------------
template <class T, bool COLFAST, class Ld, class St>
__global__ void __launch_bounds__(256) dft_cols_kernel(DftTab<T> tb, int sign, int ncols, int nb, Ld ld, St st) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smraw);
  cx<T>* scr = buf + (size_t)nb * tb.P;
  const int N = tb.N, P = tb.P;
  for (int c0 = blockIdx.x * nb; c0 < ncols; c0 += gridDim.x * nb) {
    for (int t = threadIdx.x; t < nb * N; t += blockDim.x) {
      int b, j;
      if (COLFAST) { b = t % nb; j = t / nb; } else { b = t / N; j = t % N; }
      const int c = c0 + b;
      buf[(size_t)b * P + j] = (c < ncols) ? ld(c, j) : mk<T>(0, 0);
    }
    __syncthreads();
    cx<T>* r = dft_bluestein(buf, scr, nb, tb, sign);
    for (int t = threadIdx.x; t < nb * N; t += blockDim.x) {
      int b, k;
      if (COLFAST) { b = t % nb; k = t / nb; } else { b = t / N; k = t % N; }
      const int c = c0 + b;
      if (c < ncols) st(c, k, r[(size_t)b * P + k]);
    }
    __syncthreads();
    if (r != buf) {  // keep buf as the load target of the next round
      cx<T>* s = buf; buf = scr; scr = s;
    }
  }
}

// ---------------------------------------------------------------------------
// Loaders / storers
// ---------------------------------------------------------------------------

// Synthesis over beta of a folded column X[m'][c], m' = 0..K-1 (row stride C):
// z_{m' mod N} = X~_{m'} e^{i m' pi/N}, X~_{-m'} = (-1)^{m+n+extra} X~_{m'}.
template <class T>
struct LdBetaSynth {
  const cx<T>* X; int C, K, N; ColSet cs;
  __device__ cx<T> operator()(int c, int j) const {
    int mp = (j < K) ? j : j - N;
    int a = mp < 0 ? -mp : mp;
    cx<T> v = X[(size_t)a * C + c];
    if (mp < 0 && ((cs.m_of(c) + cs.n_of(c) + cs.extra) & 1)) v = mk(-v.re, -v.im);
    T s, co;
    if (sizeof(T) == 8) { double sd, cd; sincospi((double)mp / (double)N, &sd, &cd); s = (T)sd; co = (T)cd; }
    else { float sf, cf; sincospif((float)mp / (float)N, &sf, &cf); s = (T)sf; co = (T)cf; }
    return v * mk(co, s);
  }
};
// keep k < Kout, Y[k][c]
template <class T>
struct StRows {
  cx<T>* Y; int C, Kout;
  __device__ void operator()(int c, int k, cx<T> v) const { if (k < Kout) Y[(size_t)k * C + c] = v; }
};

// Ring inverse, step over n: row (b, mi) of Xb (Nc contiguous) -> T[b][mi][g].
template <class T>
struct LdRingN {
  const cx<T>* Xb; int Nc, n0, nstep, N;
  __device__ cx<T> operator()(int c, int j) const {
    // j = n mod N; find ni with n0 + nstep*ni == n
    int n = (j <= (N - 1) / 2) ? j : j - N;
    int d = n - n0;
    if (d < 0 || d % nstep) return mk<T>(0, 0);
    int ni = d / nstep;
    if (ni >= Nc) return mk<T>(0, 0);
    return Xb[(size_t)c * Nc + ni];
  }
};
template <class T>
struct StContig {  // out[c][k], k < N
  cx<T>* out; int N;
  __device__ void operator()(int c, int k, cx<T> v) const { out[(size_t)c * N + k] = v; }
};

// Ring inverse, step over m: column (b, g) of T[b][mi][g] -> W[b][a][g].
// real: Hermitian completion z_{N-m} = conj(z_m), output real part.
template <class T>
struct LdRingM {
  const cx<T>* Tb; int Mc, m0, N; bool real;
  __device__ cx<T> operator()(int c, int j) const {
    const int b = c / N, g = c % N;
    const cx<T>* base = Tb + (size_t)b * Mc * N + g;
    int m = (j <= (N - 1) / 2) ? j : j - N;
    if (real) {
      if (m >= 0) return base[(size_t)m * N];
      return conj(base[(size_t)(-m) * N]);
    }
    int mi = m - m0;
    if (mi < 0 || mi >= Mc) return mk<T>(0, 0);
    return base[(size_t)mi * N];
  }
};
template <class T, class OutT>
struct StW {  // W[b][a][g] in OutT, real or complex
  OutT* W; int N; bool real;
  __device__ void operator()(int c, int k, cx<T> v) const {
    const int b = c / N, g = c % N;
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
  __device__ void operator()(int c, int k, cx<T> v) const {
    int n = (k <= (N - 1) / 2) ? k : k - N;
    int d = n - n0;
    if (d < 0 || d % nstep) return;
    int ni = d / nstep;
    if (ni < Nc) U[(size_t)c * Nc + ni] = v * scale;
  }
};
// Ring forward, step over a: column (b, ni) of U[b][a][ni] -> Xb[b][mi][ni].
template <class T>
struct LdRingA {
  const cx<T>* U; int Nc, N;
  __device__ cx<T> operator()(int c, int j) const {
    const int b = c / Nc, ni = c % Nc;
    return U[((size_t)b * N + j) * Nc + ni];
  }
};
template <class T>
struct StRingA {
  cx<T>* Xb; int Mc, m0, Nc, N; T scale;
  __device__ void operator()(int c, int k, cx<T> v) const {
    const int b = c / Nc, ni = c % Nc;
    int m = (k <= (N - 1) / 2) ? k : k - N;
    int mi = m - m0;
    if (mi >= 0 && mi < Mc) Xb[((size_t)b * Mc + mi) * Nc + ni] = v * scale;
  }
};

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
  __device__ void operator()(int c, int k, cx<T> v) const {
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
  template <class T> __device__ void operator()(int c, int k, cx<T> v) const {
    const size_t idx = (size_t)c * N + k;
    if (real) map[idx] = (double)v.re;
    else { map[2 * idx] = (double)v.re; map[2 * idx + 1] = (double)v.im; }
  }
};

// ---------------------------------------------------------------------------
// Exact quadrature over beta (Eqs. TildaFmn, Fmnmp, gmnmp), folded onto m' >= 0:
// per column c: extend the Lb ring values to 2Lb-1 with (-1)^{m+n+extra}, DFT
// (sign -1, half-sample phase e^{-i m'' pi/N}/N), correlate with the weights w
// (precomputed transform of v[t] = w(-t) on Q points), fold
// Yhat_{m'} = Y_{m'} + (-1)^{m+n+extra} Y_{-m'} (m' > 0), and multiply by
// scale * i^{m*pa + n*pb + pc}. In: Xb[b][c] (b < Lb); out: Y[m'][c] (m' < Lb).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) beta_quad_kernel(DftTab<T> tb, CorrTab<T> ct, int ncols, int nb, int Lb,
                                                       const cx<T>* __restrict__ Xb, cx<T>* __restrict__ Y,
                                                       ColSet cs, T scale, int pa, int pb, int pc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = tb.N, P = tb.P, Q = ct.Q;
  const int S = P > Q ? P : Q;
  cx<T>* buf = reinterpret_cast<cx<T>*>(smraw);
  cx<T>* scr = buf + (size_t)nb * S;
  for (int c0 = blockIdx.x * nb; c0 < ncols; c0 += gridDim.x * nb) {
    // gather + extension
    for (int t = threadIdx.x; t < nb * N; t += blockDim.x) {
      const int b = t % nb, j = t / nb, c = c0 + b;
      cx<T> v = mk<T>(0, 0);
      if (c < ncols) {
        if (j < Lb) v = Xb[(size_t)j * ncols + c];
        else {
          v = Xb[(size_t)(N - 1 - j) * ncols + c];
          if ((cs.m_of(c) + cs.n_of(c) + cs.extra) & 1) v = mk(-v.re, -v.im);
        }
      }
      buf[(size_t)b * P + j] = v;
    }
    __syncthreads();
    cx<T>* r = dft_bluestein(buf, scr, nb, tb, -1);
    cx<T>* o = (r == buf) ? scr : buf;
    // u_{m''} at index m'' mod Q, times e^{-i m'' pi/N}/N
    for (int t = threadIdx.x; t < nb * Q; t += blockDim.x) {
      const int b = t / Q, q = t % Q;
      int mpp = (q < Lb) ? q : q - Q;  // candidate m''
      cx<T> v = mk<T>(0, 0);
      if (mpp > -Lb && mpp < Lb) {
        const int k = (mpp >= 0) ? mpp : mpp + N;
        v = r[(size_t)b * P + k];
        T s, co;
        if (sizeof(T) == 8) { double sd, cd; sincospi(-(double)mpp / (double)N, &sd, &cd); s = (T)sd; co = (T)cd; }
        else { float sf, cf; sincospif(-(float)mpp / (float)N, &sf, &cf); s = (T)sf; co = (T)cf; }
        v = v * mk(co * ((T)1 / (T)N), s * ((T)1 / (T)N));
      }
      o[(size_t)b * Q + q] = v;
    }
    __syncthreads();
    cx<T>* u = fft_pow2(o, r, Q, nb, ct.tw, -1);
    for (int t = threadIdx.x; t < nb * Q; t += blockDim.x) u[t] = u[t] * ct.what[t % Q];
    __syncthreads();
    cx<T>* y = fft_pow2(u, (u == o) ? r : o, Q, nb, ct.tw, +1);
    // fold and store
    for (int t = threadIdx.x; t < nb * Lb; t += blockDim.x) {
      const int b = t % nb, mp = t / nb, c = c0 + b;
      if (c >= ncols) continue;
      const int m = cs.m_of(c), n = cs.n_of(c);
      cx<T> v = y[(size_t)b * Q + mp];
      if (mp > 0) {
        cx<T> w = y[(size_t)b * Q + (Q - mp)];
        if ((m + n + cs.extra) & 1) v = v - w; else v = v + w;
      }
      v = mul_ipow(v * scale, imod(m * pa + n * pb + pc, 4));
      Y[(size_t)mp * ncols + c] = v;
    }
    __syncthreads();
  }
}

}  // namespace crv
