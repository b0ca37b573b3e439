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
  int extra;    // added to m+n in parities and phases (spin for the SHT)
  FastDiv fNc;  // division by Nc
  __device__ __forceinline__ int m_of(int c) const { return m0 + (int)fNc.div((uint32_t)c); }
  __device__ __forceinline__ int n_of(int c) const { return n0 + nstep * (int)fNc.mod((uint32_t)c); }
  // parity of m + n + extra for column c
  __device__ __forceinline__ int par(int c) const {
    const uint32_t q = fNc.div((uint32_t)c);
    const int m = m0 + (int)q, n = n0 + nstep * (int)((uint32_t)c - q * (uint32_t)Nc);
    return (m + n + extra) & 1;
  }
};

// ---------------------------------------------------------------------------
// Batched DFTs of length N (Bluestein, see fft.cuh). A block holds G groups of
// P/8 threads; each group transforms one sequence at a time.
//
// rows_kernel: sequence c is gathered by ld(c, j), j < N, typically a contiguous
//   row, so each group loads its own row (coalesced along j).
// cols_kernel: consecutive sequences are adjacent in memory (columns); the block
//   stages a tile of Gc = G*cpg columns in shared memory, loading and storing with
//   the column index fastest (coalesced), and each group transforms cpg of them.
// Storers get st(c, k, X_k, X_{(N-k) mod N}) for every k < N (the second value
// serves the real-pair unpacking) and decide which outputs to keep.
// ---------------------------------------------------------------------------
template <class T, class Ld, class St>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) rows_kernel(DftTab<T> tb, int sign, int nrows, Ld ld, St st) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = tb.N, P = tb.P, Tt = P >> 3, PL = padded_len(P);
  const int G = blockDim.x / Tt, g = threadIdx.x / Tt, tt = threadIdx.x % Tt;
  cx<T>* buf = reinterpret_cast<cx<T>*>(smraw) + (size_t)g * PL;
  for (int r0 = blockIdx.x * G; r0 < nrows; r0 += gridDim.x * G) {
    const int row = r0 + g;
    const bool valid = row < nrows;
    for (int j = tt; j < P; j += Tt) {
      cx<T> v = mk<T>(0, 0);
      if (valid && j < N) v = ld(row, j) * chirp_of(tb, j, sign);
      buf[padi(j)] = v;
    }
    __syncthreads();
    bluestein_conv(buf, tb, sign, tt);
    if (valid) {
      for (int k = tt; k < N; k += Tt) {
        const int kn = (k == 0) ? 0 : N - k;
        st(row, k, buf[padi(k)] * chirp_of(tb, k, sign), buf[padi(kn)] * chirp_of(tb, kn, sign));
      }
    }
    __syncthreads();
  }
}

template <class T, class Ld, class St>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) cols_kernel(DftTab<T> tb, int sign, int ncols, int cpg,
                                                                          FastDiv fgc, Ld ld, St st) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = tb.N, P = tb.P, Tt = P >> 3, PL = padded_len(P);
  const int G = blockDim.x / Tt, g = threadIdx.x / Tt, tt = threadIdx.x % Tt;
  const int Gc = G * cpg;
  const int CS = N | 1;                                     // odd column stride: no bank conflicts
  cx<T>* tile = reinterpret_cast<cx<T>*>(smraw);          // [Gc][CS]
  cx<T>* buf = tile + (size_t)Gc * CS + (size_t)g * PL;    // per group work buffer
  for (int c0 = blockIdx.x * Gc; c0 < ncols; c0 += gridDim.x * Gc) {
    for (int t = threadIdx.x; t < Gc * N; t += blockDim.x) {
      const int j = (int)fgc.div(t), b = t - j * Gc, c = c0 + b;
      tile[(size_t)b * CS + j] = (c < ncols) ? ld(c, j) : mk<T>(0, 0);
    }
    __syncthreads();
    for (int q = 0; q < cpg; ++q) {
      const int b = g * cpg + q;
      cx<T>* col = tile + (size_t)b * CS;
      for (int j = tt; j < P; j += Tt) buf[padi(j)] = (j < N) ? col[j] * chirp_of(tb, j, sign) : mk<T>(0, 0);
      __syncthreads();
      bluestein_conv(buf, tb, sign, tt);
      for (int k = tt; k < N; k += Tt) col[k] = buf[padi(k)] * chirp_of(tb, k, sign);
      __syncthreads();
    }
    for (int t = threadIdx.x; t < Gc * N; t += blockDim.x) {
      const int k = (int)fgc.div(t), b = t - k * Gc, c = c0 + b;
      if (c < ncols) {
        const int kn = (k == 0) ? 0 : N - k;
        st(c, k, tile[(size_t)b * CS + k], tile[(size_t)b * CS + kn]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Loaders / storers
// ---------------------------------------------------------------------------

// Synthesis over beta of a folded column X[m'][c], m' = 0..K-1 (row stride C):
// z_{m' mod N} = X~_{m'} e^{i m' pi/N}, X~_{-m'} = (-1)^{m+n+extra} X~_{m'}.
template <class T>
struct LdBetaSynth {
  const cx<T>* X; int C, K, N; ColSet cs; const cx<T>* hphase;
  __device__ cx<T> operator()(int c, int j) const {
    int mp = (j < K) ? j : j - N;
    int a = mp < 0 ? -mp : mp;
    cx<T> v = X[(size_t)a * C + c];
    if (mp < 0 && cs.par(c)) v = mk(-v.re, -v.im);
    return v * hphase[j];
  }
};
// keep k < Kout, Y[k][c]
template <class T>
struct StRows {
  cx<T>* Y; int C, Kout;
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const { if (k < Kout) Y[(size_t)k * C + c] = v; }
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
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const { out[(size_t)c * N + k] = v; }
};

// Ring inverse, step over m: column (b, g) of T[b][mi][g] -> W[b][a][g].
// real: Hermitian completion z_{N-m} = conj(z_m), output real part.
template <class T>
struct LdRingM {
  const cx<T>* Tb; int Mc, m0, N; bool real; FastDiv fN;
  __device__ cx<T> operator()(int c, int j) const {
    const int b = (int)fN.div(c), g = c - b * N;
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
    if (d < 0 || d % nstep) return;
    int ni = d / nstep;
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
  cx<T>* Xb; int Mc, m0, Nc, N; T scale; FastDiv fNc;
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const {
    const int b = (int)fNc.div(c), ni = c - b * Nc;
    int m = (k <= (N - 1) / 2) ? k : k - N;
    int mi = m - m0;
    if (mi >= 0 && mi < Mc) Xb[((size_t)b * Mc + mi) * Nc + ni] = v * scale;
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
};
template <class T>
struct StRingNPair {
  cx<T>* U; int Nc, n0, nstep, N, nrows; T scale;
  __device__ void operator()(int c, int k, cx<T> z, cx<T> zn) const {
    int n = (k <= (N - 1) / 2) ? k : k - N;
    int d = n - n0;
    if (d < 0 || d % nstep) return;
    int ni = d / nstep;
    if (ni >= Nc) return;
    const T h = scale * (T)0.5;
    const cx<T> a = mk<T>((z.re + zn.re) * h, (z.im - zn.im) * h);   // (z + conj zn)/2
    const cx<T> b = mk<T>((z.im + zn.im) * h, (zn.re - z.re) * h);   // (z - conj zn)/(2i)
    U[(size_t)(2 * c) * Nc + ni] = a;
    if (2 * c + 1 < nrows) U[(size_t)(2 * c + 1) * Nc + ni] = b;
  }
};
// Inverse over m with Hermitian input and real output: columns g = 2c, 2c+1 packed.
template <class T>
struct LdRingMPair {
  const cx<T>* Tb; int Mc, N, npair; FastDiv fP;
  __device__ cx<T> operator()(int c, int j) const {
    const int b = (int)fP.div(c), gp = c - b * npair, g1 = 2 * gp, g2 = g1 + 1;
    const cx<T>* base = Tb + (size_t)b * Mc * N;
    int m = (j <= (N - 1) / 2) ? j : j - N;
    const int am = m < 0 ? -m : m;
    cx<T> t1 = base[(size_t)am * N + g1];
    cx<T> t2 = (g2 < N) ? base[(size_t)am * N + g2] : mk<T>(0, 0);
    if (m < 0) { t1 = conj(t1); t2 = conj(t2); }
    return mk<T>(t1.re - t2.im, t1.im + t2.re);
  }
};
template <class T, class OutT>
struct StWPair {
  OutT* W; int N, npair; FastDiv fP;
  __device__ void operator()(int c, int k, cx<T> v, cx<T>) const {
    const int b = (int)fP.div(c), gp = c - b * npair, g1 = 2 * gp, g2 = g1 + 1;
    const size_t idx = ((size_t)b * N + k) * N;
    W[idx + g1] = (OutT)v.re;
    if (g2 < N) W[idx + g2] = (OutT)v.im;
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
// Exact quadrature over beta (Eqs. TildaFmn, Fmnmp, gmnmp), folded onto m' >= 0:
// per column c: extend the Lb ring values to 2Lb-1 with (-1)^{m+n+extra}, DFT
// (sign -1, half-sample phase e^{-i m'' pi/N}/N), correlate with the weights w
// (precomputed transform of v[t] = w(-t) on Q = P points), fold
// Yhat_{m'} = Y_{m'} + (-1)^{m+n+extra} Y_{-m'} (m' > 0), and multiply by
// scale * i^{m*pa + n*pb + pc}. In: Xb[b][c] (b < Lb); out: Y[m'][c] (m' < Lb).
// Same tiling as cols_kernel.
// ---------------------------------------------------------------------------
// e^{-i m pi/N} / N
template <class T>
__device__ __forceinline__ cx<T> half_phase(int m, int N, T invN) {
  T s, co;
  if (sizeof(T) == 8) { double sd, cd; sincospi(-(double)m / (double)N, &sd, &cd); s = (T)sd; co = (T)cd; }
  else { float sf, cf; sincospif(-(float)m / (float)N, &sf, &cf); s = (T)sf; co = (T)cf; }
  return mk(co * invN, s * invN);
}

template <class T>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) beta_quad_kernel(DftTab<T> tb, CorrTab<T> ct, int ncols, int cpg, int Lb,
                                                       FastDiv fgc, const cx<T>* __restrict__ Xb, cx<T>* __restrict__ Y,
                                                       ColSet cs, T scale, int pa, int pb, int pc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = tb.N, P = tb.P, Q = ct.Q, Tt = P >> 3, PL = padded_len(P);
  const int G = blockDim.x / Tt, g = threadIdx.x / Tt, tt = threadIdx.x % Tt;
  const int Gc = G * cpg;
  const int CS = Lb | 1;                           // odd column stride: no bank conflicts
  cx<T>* tile = reinterpret_cast<cx<T>*>(smraw);  // [Gc][CS]
  cx<T>* buf = tile + (size_t)Gc * CS + (size_t)g * PL;
  const T invN = (T)1 / (T)N;
  for (int c0 = blockIdx.x * Gc; c0 < ncols; c0 += gridDim.x * Gc) {
    for (int t = threadIdx.x; t < Gc * Lb; t += blockDim.x) {
      const int j = (int)fgc.div(t), b = t - j * Gc, c = c0 + b;
      tile[(size_t)b * CS + j] = (c < ncols) ? Xb[(size_t)j * ncols + c] : mk<T>(0, 0);
    }
    __syncthreads();
    for (int q = 0; q < cpg; ++q) {
      const int b = g * cpg + q, c = c0 + b;
      cx<T>* col = tile + (size_t)b * CS;
      const int par = (c < ncols) ? cs.par(c) : 0;
      for (int j = tt; j < P; j += Tt) {
        cx<T> v = mk<T>(0, 0);
        if (j < Lb) v = col[j];
        else if (j < N) { v = col[N - 1 - j]; if (par) v = mk(-v.re, -v.im); }
        buf[padi(j)] = v * chirp_of(tb, j < N ? j : 0, -1);
      }
      __syncthreads();
      bluestein_conv(buf, tb, -1, tt);
      // u_{m''} at index m'' mod Q: D_{m'' mod N} h_k e^{-i m'' pi/N} / N, in place in two
      // phases: the negative m'' (sources k in [Lb, N), targets q >= N, disjoint), then
      // m'' >= 0 (same index) and the zero gap.
      for (int qi = Q - Lb + 1 + tt; qi < Q; qi += Tt) {
        const int mpp = qi - Q, k = mpp + N;
        buf[padi(qi)] = buf[padi(k)] * chirp_of(tb, k, -1) * (conj(tb.hphase[k]) * invN);
      }
      __syncthreads();
      for (int qi = tt; qi <= Q - Lb; qi += Tt)
        buf[padi(qi)] = (qi < Lb) ? buf[padi(qi)] * chirp_of(tb, qi, -1) * (conj(tb.hphase[qi]) * invN) : mk<T>(0, 0);
      __syncthreads();
      fft_p2(buf, Q, ct.tw, -1, tt);
      for (int i = tt; i < Q; i += Tt) buf[padi(i)] = buf[padi(i)] * ct.what[i];
      __syncthreads();
      fft_p2(buf, Q, ct.tw, +1, tt);
      if (c < ncols) {
        const int m = cs.m_of(c), n = cs.n_of(c);
        const int ph = imod(m * pa + n * pb + pc, 4);
        for (int mp = tt; mp < Lb; mp += Tt) {
          cx<T> v = buf[padi(mp)];
          if (mp > 0) {
            const cx<T> w = buf[padi(Q - mp)];
            v = par ? v - w : v + w;
          }
          col[mp] = mul_ipow(v * scale, ph);
        }
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < Gc * Lb; t += blockDim.x) {
      const int mp = (int)fgc.div(t), b = t - mp * Gc, c = c0 + b;
      if (c < ncols) Y[(size_t)mp * ncols + c] = tile[(size_t)b * CS + mp];
    }
    __syncthreads();
  }
}

}  // namespace crv
