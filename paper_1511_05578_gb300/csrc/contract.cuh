// Delta contractions of the Wigner transforms and the spin SHT (CUDA-core form).
//
// Analysis (inverse Wigner, Eq. inverse_Fmnmp in general-n form with the
// coefficients of Eq. wav_harmonic_coeff folded in):
//   X_{m n m'} = i^{n-m} sum_l Delta^l_{m'm} Delta^l_{m'n} f_lm Psi_ln,   m' >= 0.
// Per m' this is a product U(m') V(m') with U_{m,l} = Delta^l_{m'm} f_lm and
// V_{l,n} = Delta^l_{m'n} Psi_ln, both built on the fly from the quarter Delta table.
//
// Synthesis (forward Wigner, Eq. flml in general-n form, then the n-sum of Eq.
// wav_synthesis_harmonic):
//   f_lm += sum_{m'>=0} Delta^l_{m'm} sum_n (Delta^l_{m'n} Psi_ln) Y'_{m n m'},
// where Y' already carries i^{m-n}. Per m' the inner sum is a product Y'(m') V(m')^T;
// the outer sum over m' accumulates in FP64 registers and is flushed with FP64
// atomics once per block.
#pragma once
#include "transforms.cuh"

namespace crv {

// Delta^l_{a,b} for a >= 0 and any b, from the quarter table Q[a][l][|b|].
template <class T>
__device__ __forceinline__ T delta_q(const T* __restrict__ Q, int Lmax, int a, int l, int b) {
  const int ab = b < 0 ? -b : b;
  T v = Q[((size_t)a * Lmax + l) * Lmax + ab];
  if (b < 0 && ((l + a) & 1)) v = -v;
  return v;
}

// ---------------------------------------------------------------------------
// Analysis contraction. Block tile 32 (m) x 64 (n), K-step 16, 256 threads,
// each thread 2 x 4 outputs. grid = (ceil(Nc/64), ceil(Mc/32), Lb).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) contract_analysis_kernel(const T* __restrict__ Q, int Lmax,
                                                                const cx<double>* __restrict__ flm,
                                                                const T* __restrict__ psi, int Lb, ColSet cs,
                                                                cx<T>* __restrict__ X) {
  constexpr int TM = 32, TN = 64, TK = 16;
  __shared__ cx<T> As[TK][TM];
  __shared__ T Bs[TK][TN];
  const int N = 2 * Lb - 1;
  const int mp = blockIdx.z;
  const int mi0 = blockIdx.y * TM, ni0 = blockIdx.x * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // smallest |m|, |n| in the tile -> first useful l
  int mlo = cs.m0 + mi0, mhi = cs.m0 + min(mi0 + TM, cs.Mc) - 1;
  int nlo = cs.n0 + cs.nstep * ni0, nhi = cs.n0 + cs.nstep * (min(ni0 + TN, cs.Nc) - 1);
  int amin = (mlo <= 0 && mhi >= 0) ? 0 : min(abs(mlo), abs(mhi));
  int bmin = (nlo <= 0 && nhi >= 0) ? 0 : min(abs(nlo), abs(nhi));
  int lstart = max(mp, max(amin, bmin));
  cx<T> acc[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<T>(0, 0);
  for (int l0 = lstart; l0 < Lb; l0 += TK) {
    // A tile: 512 complex entries, 2 per thread
    for (int t = threadIdx.x; t < TK * TM; t += 256) {
      const int k = t / TM, i = t % TM, l = l0 + k, mi = mi0 + i;
      cx<T> v = mk<T>(0, 0);
      if (l < Lb && mi < cs.Mc) {
        const int m = cs.m0 + mi;
        if (abs(m) <= l) {
          const cx<double> f = flm[l * l + l + m];
          const T d = delta_q(Q, Lmax, mp, l, m);
          v = mk<T>(d * (T)f.re, d * (T)f.im);
        }
      }
      As[k][i] = v;
    }
    for (int t = threadIdx.x; t < TK * TN; t += 256) {
      const int k = t / TN, j = t % TN, l = l0 + k, ni = ni0 + j;
      T v = 0;
      if (l < Lb && ni < cs.Nc) {
        const int n = cs.n0 + cs.nstep * ni;
        if (abs(n) <= l) v = delta_q(Q, Lmax, mp, l, n) * psi[(size_t)l * N + (n + Lb - 1)];
      }
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      const cx<T> a0 = As[k][ty * 2], a1 = As[k][ty * 2 + 1];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const T b = Bs[k][tx * 4 + j];
        acc[0][j].re += a0.re * b; acc[0][j].im += a0.im * b;
        acc[1][j].re += a1.re * b; acc[1][j].im += a1.im * b;
      }
    }
    __syncthreads();
  }
  const size_t plane = cs.pitch();
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int mi = mi0 + ty * 2 + i;
    if (mi >= cs.Mc) continue;
    const int m = cs.m0 + mi;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ni = ni0 + tx * 4 + j;
      if (ni >= cs.Nc) continue;
      const int n = cs.n0 + cs.nstep * ni;
      X[(size_t)mp * plane + cs.col(mi, ni)] = mul_ipow(acc[i][j], imod(n - m, 4));
    }
  }
}

// ---------------------------------------------------------------------------
// Synthesis contraction. Block tile 32 (m) x 32 (l), 256 threads, 2 x 2 outputs
// per thread, K-step 16 over n, a chunk of m' values per block.
// grid = (ceil(Lb/32), ceil(Mc/32), ceil(Lb/mchunk)).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) contract_synthesis_kernel(const T* __restrict__ Q, int Lmax,
                                                                 const cx<T>* __restrict__ Y,
                                                                 const T* __restrict__ psi, int Lb, ColSet cs,
                                                                 int mchunk, cx<double>* __restrict__ flm) {
  constexpr int TM = 32, TL = 32, TK = 16;
  __shared__ cx<T> Ys[TM][TK + 1];
  __shared__ T Vs[TK][TL];
  const int N = 2 * Lb - 1;
  const int l0 = blockIdx.x * TL, mi0 = blockIdx.y * TM;
  const int lhi = min(l0 + TL, Lb) - 1;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int mlo = cs.m0 + mi0, mhi = cs.m0 + min(mi0 + TM, cs.Mc) - 1;
  const int amin = (mlo <= 0 && mhi >= 0) ? 0 : min(abs(mlo), abs(mhi));
  if (amin > lhi) return;
  // n range with |n| <= lhi
  int ni_lo = 0, ni_hi = cs.Nc;  // [ni_lo, ni_hi)
  {
    int nmin = -lhi;
    int d = nmin - cs.n0;
    ni_lo = d <= 0 ? 0 : (d + cs.nstep - 1) / cs.nstep;
    int dmax = lhi - cs.n0;
    ni_hi = dmax < 0 ? 0 : min(cs.Nc, dmax / cs.nstep + 1);
  }
  cx<double> facc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i) { facc[i][0] = mk(0.0, 0.0); facc[i][1] = mk(0.0, 0.0); }
  const size_t plane = cs.pitch();
  const int mp_end = min((int)(blockIdx.z + 1) * mchunk, lhi + 1);
  for (int mp = blockIdx.z * mchunk; mp < mp_end; ++mp) {
    cx<T> z[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) { z[i][0] = mk<T>(0, 0); z[i][1] = mk<T>(0, 0); }
    for (int nk = ni_lo; nk < ni_hi; nk += TK) {
      for (int t = threadIdx.x; t < TM * TK; t += 256) {
        const int i = t / TK, k = t % TK, mi = mi0 + i, ni = nk + k;
        Ys[i][k] = (mi < cs.Mc && ni < ni_hi) ? Y[(size_t)mp * plane + cs.col(mi, ni)] : mk<T>(0, 0);
      }
      for (int t = threadIdx.x; t < TK * TL; t += 256) {
        const int k = t / TL, j = t % TL, ni = nk + k, l = l0 + j;
        T v = 0;
        if (ni < ni_hi && l < Lb && l >= mp) {
          const int n = cs.n0 + cs.nstep * ni;
          if (abs(n) <= l) v = delta_q(Q, Lmax, mp, l, n) * psi[(size_t)l * N + (n + Lb - 1)];
        }
        Vs[k][j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < TK; ++k) {
        const cx<T> y0 = Ys[ty * 2][k], y1 = Ys[ty * 2 + 1][k];
        const T v0 = Vs[k][tx * 2], v1 = Vs[k][tx * 2 + 1];
        z[0][0].re += y0.re * v0; z[0][0].im += y0.im * v0;
        z[0][1].re += y0.re * v1; z[0][1].im += y0.im * v1;
        z[1][0].re += y1.re * v0; z[1][0].im += y1.im * v0;
        z[1][1].re += y1.re * v1; z[1][1].im += y1.im * v1;
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int mi = mi0 + ty * 2 + i;
      if (mi >= cs.Mc) continue;
      const int m = cs.m0 + mi;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int l = l0 + tx * 2 + j;
        if (l >= Lb || l < mp || abs(m) > l) continue;
        const double d = (double)delta_q(Q, Lmax, mp, l, m);
        facc[i][j].re += d * (double)z[i][j].re;
        facc[i][j].im += d * (double)z[i][j].im;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int mi = mi0 + ty * 2 + i;
    if (mi >= cs.Mc) continue;
    const int m = cs.m0 + mi;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int l = l0 + tx * 2 + j;
      if (l >= Lb || abs(m) > l) continue;
      atomicAdd(&flm[l * l + l + m].re, facc[i][j].re);
      atomicAdd(&flm[l * l + l + m].im, facc[i][j].im);
    }
  }
}

// ---------------------------------------------------------------------------
// Unrotated curvelets (Sec. III-A-1, plans with CRV_F_UNROTATED). The Wigner coefficients
// of W~ vanish unless |n| = l (Eq. curvelet_Wigner_property), so each Delta contraction
// keeps a single term:
//   analysis  (Eq. inverse_Fmnmp):    X_{m n m'} = i^{n-m} Delta^{|n|}_{m'm} Delta^{|n|}_{m'n} f_{|n| m} Psi~_{|n| n}
//   synthesis (Eq. flml with n = +-l): f_lm += sum_{m'>=0} Delta^l_{m'm} sum_{n=+-l} Delta^l_{m'n} Psi~_ln Y'_{m n m'}
// (Y' carries i^{m-n}), O(L^3) per scale and bound by the volume traffic. The planes hold
// every n (nstep = 1), pair-interleaved as everywhere.
// ---------------------------------------------------------------------------
constexpr int UA_PAIRS = 8, UA_N = 64;
// m' planes per block of the analysis fill and per step of the synthesis loop
template <class T> struct UnrotPlanes { static constexpr int value = sizeof(T) == 4 ? 4 : 2; };

// A block covers UnrotPlanes (m, n) planes m' from blockIdx.z * UnrotPlanes on, and
// UA_PAIRS column pairs (m, m+1) x UA_N values of n. Phase 1 forms the products with m
// fastest (coalesced rows Q[m'][l][|m|] and f_lm, the latter once for all planes); phase 2
// writes them in column order (per pair row, 2 UA_N contiguous columns).
// Column pairs (m, m+1) at n that are zero as a whole (|n| < nlo, the first l of the support
// of kappa^(j), or both |m|, |m+1| > |n|) are not written: the beta transforms skip them.
// Every other column of the plane is written, zeros included.
// grid = (ceil(Nc / UA_N), ceil(ceil(Mc/2) / UA_PAIRS), ceil(Lb / UnrotPlanes)).
template <class T>
__global__ void __launch_bounds__(256) unrot_analysis_kernel(const T* __restrict__ Q, int Lmax,
                                                             const cx<double>* __restrict__ flm,
                                                             const T* __restrict__ psi, int Lb, ColSet cs,
                                                             int nlo, cx<T>* __restrict__ X) {
  constexpr int MPB = UnrotPlanes<T>::value, E = UA_N * 2 * UA_PAIRS / 256;
  __shared__ cx<T> S[MPB][UA_N][2 * UA_PAIRS + 1];
  const int N = 2 * Lb - 1, mpb = blockIdx.z * MPB;
  const int pi0 = blockIdx.y * UA_PAIRS, mi0 = 2 * pi0, ni0 = blockIdx.x * UA_N;
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int e = t + 256 * k, nl = e / (2 * UA_PAIRS), ml = e % (2 * UA_PAIRS);
    const int mi = mi0 + ml, ni = ni0 + nl;
    const int m = cs.m0 + mi, n = cs.n0 + ni;
    const int l = n < 0 ? -n : n, am = m < 0 ? -m : m;
    cx<T> base = mk<T>(0, 0);
    T ps = 0;
    const bool live = mi < cs.Mc && ni < cs.Nc && l >= am && l >= mpb;
    if (live) ps = psi[(size_t)l * N + (n + Lb - 1)];
    if (ps != (T)0) {
      const cx<double> f = flm[l * l + l + m];
      base = mul_ipow(mk<T>(ps * (T)f.re, ps * (T)f.im), imod(n - m, 4));
    }
    T d[MPB];
#pragma unroll
    for (int q = 0; q < MPB; ++q) {
      const int mp = mpb + q;
      d[q] = (ps != (T)0 && mp < Lb && l >= mp) ? delta_q(Q, Lmax, mp, l, m) * delta_q(Q, Lmax, mp, l, n) : (T)0;
    }
#pragma unroll
    for (int q = 0; q < MPB; ++q) S[q][nl][ml] = base * d[q];
  }
  __syncthreads();
  const int npairs = (cs.Mc + 1) >> 1;
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int e = t + 256 * k, r = e / (2 * UA_N), w = e % (2 * UA_N), nl = w >> 1, par = w & 1;
    const int ni = ni0 + nl;
    if (pi0 + r >= npairs || ni >= cs.Nc) continue;
    const int n = cs.n0 + ni, an = n < 0 ? -n : n, ma = cs.m0 + 2 * (pi0 + r), mb = ma + 1;
    const bool live = an >= nlo && ((ma < 0 ? -ma : ma) <= an || (mi0 + 2 * r + 1 < cs.Mc && (mb < 0 ? -mb : mb) <= an));
    if (!live) continue;
    const size_t c = ((size_t)(pi0 + r) * cs.Nc + ni) * 2 + par;
#pragma unroll
    for (int q = 0; q < MPB; ++q)
      if (mpb + q < Lb) X[(size_t)(mpb + q) * cs.pitch() + c] = S[q][nl][2 * r + par];
  }
}

constexpr int US_L = 32, US_PAIRS = 8, US_MPC = 128;

// Synthesis: a block covers US_L values of l (both n = +l and n = -l) x US_PAIRS column
// pairs and a chunk of US_MPC values of m', UnrotPlanes at a time: the rows Delta^l_{m'm} of
// the tile pass through shared memory (loaded m fastest), the Y' columns are read in column
// order; thread slot k holds n = +l and slot k + 2 the same (l, m) with n = -l. Products are
// summed in T, flushed to FP64 every 32 m'; the chunk's sums go to P[chunk][l*l + l + m] for
// every l < Lb, m in the m-set, |m| <= l (zeros included), and unrot_reduce_kernel adds the
// chunks in order. Columns with l = |n| < nlo (below the support of kappa^(j), Psi~ = 0) are
// not read: the beta quadrature does not produce them.
// grid = (ceil(Lb / US_L), ceil(ceil(Mc/2) / US_PAIRS), ceil(Lb / US_MPC)).
template <class T>
__global__ void __launch_bounds__(256) unrot_synthesis_kernel(const T* __restrict__ Q, int Lmax,
                                                              const cx<T>* __restrict__ Y,
                                                              const T* __restrict__ psi, int Lb, ColSet cs,
                                                              int nlo, cx<double>* __restrict__ P) {
  constexpr int MPS = UnrotPlanes<T>::value;
  static_assert(US_MPC % MPS == 0 && 32 % MPS == 0, "plane step divides the chunk and the flush period");
  __shared__ T Dm[2][MPS][US_L][2 * US_PAIRS + 1];  // Delta^l_{m'm}
  __shared__ T Dn[2][MPS][2][US_L];                  // Delta^l_{m',+-l} Psi~_{l,+-l}
  const int N = 2 * Lb - 1;
  const int l0 = blockIdx.x * US_L, pi0 = blockIdx.y * US_PAIRS, mi0 = 2 * pi0;
  const int mp0 = blockIdx.z * US_MPC;
  const int lhi = min(l0 + US_L, Lb) - 1;
  const int mp1 = min(mp0 + US_MPC, lhi + 1);
  const size_t pitch = cs.pitch();
  const int t = threadIdx.x;
  // the thread's four slots: e = t + 256 k -> (sign, pair row r, l, parity)
  size_t col[4];
  int ll[4], ml[4];
  bool ok[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = t + 256 * k, sg = e / (US_PAIRS * 2 * US_L), r = (e / (2 * US_L)) % US_PAIRS, w = e % (2 * US_L);
    ll[k] = w >> 1;
    ml[k] = 2 * r + (w & 1);
    const int l = l0 + ll[k], mi = mi0 + ml[k], m = cs.m0 + mi;
    const int n = sg ? -l : l;
    ok[k] = l < Lb && l >= nlo && mi < cs.Mc && (m < 0 ? -m : m) <= l && !(sg && l == 0);
    col[k] = ok[k] ? ((size_t)(pi0 + r) * cs.Nc + (n - cs.n0)) * 2 + (w & 1) : 0;
  }
  cx<double> acc[4];
  cx<T> part[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) { acc[k] = mk(0.0, 0.0); part[k] = mk<T>(0, 0); }
  int it = 0;
  for (int mpb = mp0; mpb < mp1; mpb += MPS, ++it) {
    const int bf = it & 1;
    for (int e = t; e < MPS * US_L * 2 * US_PAIRS; e += 256) {
      const int q = e / (US_L * 2 * US_PAIRS), a = (e / (2 * US_PAIRS)) % US_L, b = e % (2 * US_PAIRS);
      const int mp = mpb + q, l = l0 + a, mi = mi0 + b, m = cs.m0 + mi;
      T d = 0;
      if (mp < mp1 && l < Lb && l >= mp && mi < cs.Mc && (m < 0 ? -m : m) <= l) d = delta_q(Q, Lmax, mp, l, m);
      Dm[bf][q][a][b] = d;
    }
    if (t < MPS * 2 * US_L) {
      const int q = t / (2 * US_L), sg = (t / US_L) & 1, a = t % US_L, mp = mpb + q, l = l0 + a, n = sg ? -l : l;
      T d = 0;
      if (mp < mp1 && l < Lb && l >= mp) d = delta_q(Q, Lmax, mp, l, n) * psi[(size_t)l * N + (n + Lb - 1)];
      Dn[bf][q][sg][a] = d;
    }
    __syncthreads();
    cx<T> y[MPS][4];
#pragma unroll
    for (int q = 0; q < MPS; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        y[q][k] = (ok[k] && mpb + q < mp1) ? Y[(size_t)(mpb + q) * pitch + col[k]] : mk<T>(0, 0);
#pragma unroll
    for (int q = 0; q < MPS; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const T c = Dm[bf][q][ll[k]][ml[k]] * Dn[bf][q][k >> 1][ll[k]];
        part[k].re += c * y[q][k].re;
        part[k].im += c * y[q][k].im;
      }
    if (((mpb + MPS - mp0) & 31) == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        acc[k].re += (double)part[k].re; acc[k].im += (double)part[k].im;
        part[k] = mk<T>(0, 0);
      }
    }
  }
  const int cidx = blockIdx.z;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    acc[k].re += (double)part[k].re + (double)part[k + 2].re + acc[k + 2].re;
    acc[k].im += (double)part[k].im + (double)part[k + 2].im + acc[k + 2].im;
    const int l = l0 + ll[k], mi = mi0 + ml[k], m = cs.m0 + mi;
    if (l < Lb && mi < cs.Mc && (m < 0 ? -m : m) <= l) P[(size_t)cidx * Lb * Lb + l * l + l + m] = acc[k];
  }
}

// f_lm += sum_c P[c][l*l + l + m] in chunk order, for l < Lb and m in the m-set.
static __global__ void unrot_reduce_kernel(const cx<double>* __restrict__ P, int nchunk, int Lb, int m0,
                                           cx<double>* __restrict__ flm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Lb * Lb) return;
  int l = (int)sqrt((double)i);
  if (l * l > i) --l;
  if ((l + 1) * (l + 1) <= i) ++l;
  if (i - l * l - l < m0) return;
  cx<double> s = flm[i];
  for (int c = 0; c < nchunk; ++c) s = s + P[(size_t)c * Lb * Lb + i];
  flm[i] = s;
}

// ---------------------------------------------------------------------------
// SHT contractions (FP64; O(L^3) total).
// Forward:  f_lm = sqrt((2l+1)/4pi) sum_{m'>=0} Delta^l_{m'm} Delta^l_{m',-s} G'[m'][mi]
//           (G' carries (-1)^s i^{m+s} and the folding over +-m').
// Inverse:  G[m'][mi] = (-1)^s i^{-(m+s)} sum_l sqrt((2l+1)/4pi) Delta^l_{m'm} Delta^l_{m',-s} f_lm.
// ---------------------------------------------------------------------------
static __global__ void sht_fwd_contract_kernel(const double* __restrict__ Q, int Lmax, const cx<double>* __restrict__ G,
                                        int Ls, int s, int Mc, int m0, cx<double>* __restrict__ flm) {
  const int mi = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = blockIdx.y;
  if (mi >= Mc) return;
  const int m = m0 + mi;
  if (abs(m) > l) return;
  cx<double> acc = mk(0.0, 0.0);
  if (l >= abs(s)) {
    for (int mp = 0; mp <= l; ++mp) {
      const double d = delta_q(Q, Lmax, mp, l, m) * delta_q(Q, Lmax, mp, l, -s);
      const cx<double> g = G[(size_t)mp * Mc + mi];
      acc.re += d * g.re; acc.im += d * g.im;
    }
  }
  const double nrm = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
  flm[l * l + l + m] = acc * nrm;
}

// Dynamic shared memory: Ls doubles (the normalisations sqrt((2l+1)/4pi)).
static __global__ void sht_inv_contract_kernel(const double* __restrict__ Q, int Lmax, const cx<double>* __restrict__ flm,
                                        int Ls, int s, int Mc, int m0, cx<double>* __restrict__ G) {
  extern __shared__ double nrm[];
  for (int l = threadIdx.x; l < Ls; l += blockDim.x) nrm[l] = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
  __syncthreads();
  const int mi = blockIdx.x * blockDim.x + threadIdx.x;
  const int mp = blockIdx.y;
  if (mi >= Mc) return;
  const int m = m0 + mi;
  cx<double> acc = mk(0.0, 0.0);
  int lstart = max(mp, max(abs(m), abs(s)));
  for (int l = lstart; l < Ls; ++l) {
    const double d = nrm[l] * delta_q(Q, Lmax, mp, l, m) * delta_q(Q, Lmax, mp, l, -s);
    const cx<double> f = flm[l * l + l + m];
    acc.re += d * f.re; acc.im += d * f.im;
  }
  acc = mul_ipow(acc, imod(-(m + s) + 2 * s, 4));
  G[(size_t)mp * Mc + mi] = acc;
}

// f_{l,-m} = (-1)^m conj(f_lm) for m > 0 (real signals); zero for l < |s| or l >= Lkeep.
static __global__ void flm_finish_kernel(cx<double>* __restrict__ flm, int L, int s, bool real) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L * L) return;
  const int l = (int)sqrt((double)i);
  int ll = l;
  if (ll * ll > i) --ll;
  if ((ll + 1) * (ll + 1) <= i) ++ll;
  const int m = i - ll * ll - ll;
  if (ll < abs(s)) { flm[i] = mk(0.0, 0.0); return; }
  if (real && m < 0) {
    cx<double> v = flm[ll * ll + ll - m];
    v = conj(v);
    if ((-m) & 1) v = mk(-v.re, -v.im);
    flm[i] = v;
  }
}

// c_lm = phi_l f_lm (l < Lp), packed for band limit Lp; or f_lm += phi_l c_lm.
static __global__ void scaling_apply_kernel(const double* __restrict__ phi, int Lp, const cx<double>* __restrict__ in,
                                     cx<double>* __restrict__ out, bool accumulate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Lp * Lp) return;
  int l = (int)sqrt((double)i);
  if (l * l > i) --l;
  if ((l + 1) * (l + 1) <= i) ++l;
  const cx<double> v = in[i] * phi[l];
  if (accumulate) out[i] = out[i] + v;
  else out[i] = v;
}

template <class T>
__global__ void cast_flm_kernel(const cx<double>* __restrict__ in, cx<T>* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = mk<T>((T)in[i].re, (T)in[i].im);
}

}  // namespace crv
