// Tensor-core (tcgen05, sm_103a) split-FP32 Delta contractions of the mixed path.
//
// Analysis (Eq. inverse_Fmnmp, general n, with Eq. wav_harmonic_coeff folded in), per m' >= 0:
//   D[(m, re|im)][n] = sum_l A[(m, re|im)][l] B[n][l],
//   A = Delta^l_{m'm} (Re|Im f_lm),  B = Delta^l_{m'n} Psi_ln,
//   X_{m n m'} = i^{n-m} (D_re + i D_im).
// Synthesis (Eq. flml general n, then the n-sum of Eq. wav_synthesis_harmonic), per m':
//   Z[(m, re|im)][l] = sum_n A[(m, re|im)][n] B[l][n],  A = Y'_{m n m'} (carries i^{m-n}),
//   B = Delta^l_{m'n} Psi_ln; then f_lm += sum_{m'} Delta^l_{m'm} Z_{m l m'} in FP64.
//
// Each FP32 operand x is split into TF32 hi = rna(x), lo = rna(x - hi); a K-step issues
// hi*hi + hi*lo + lo*hi into the same FP32 TMEM accumulator (split-FP32, ~2^-22 per
// product). Operands are built on the fly by all 256 threads into shared memory in the
// canonical K-major no-swizzle layout (8-row x 16-byte core matrices), double-buffered;
// one thread issues tcgen05.mma and commits to an mbarrier per stage; waits are bounded
// and set an error flag instead of hanging. The accumulator tile is 128 lanes x 128
// columns of TMEM, drained by four warps with tcgen05.ld.
#include "tc_gemm.cuh"

namespace crv {
namespace tc {

constexpr int BNC = 256;  // accumulator width of the contraction tiles

// ---------------------------------------------------------------------------
// Problems: operand builders, K ranges and epilogues
// ---------------------------------------------------------------------------
struct AnalysisProb {
  const float* Q; int Lmax; const cx<float>* flm; const float* psi; int Lb; ColSet cs; cx<float>* X;
  __device__ void tile(int& mp, int& mi0, int& n0i, int& kb, int& ke) const {
    mp = blockIdx.z; mi0 = blockIdx.y * (BM / 2); n0i = blockIdx.x * BNC;
    const int mlo = cs.m0 + mi0, mhi = cs.m0 + min(mi0 + BM / 2, cs.Mc) - 1;
    const int nlo = cs.n0 + cs.nstep * n0i, nhi = cs.n0 + cs.nstep * (min(n0i + BNC, cs.Nc) - 1);
    const int amin = (mlo <= 0 && mhi >= 0) ? 0 : min(abs(mlo), abs(mhi));
    const int bmin = (nlo <= 0 && nhi >= 0) ? 0 : min(abs(nlo), abs(nhi));
    kb = max(mp, max(amin, bmin));
    ke = Lb;
  }
  // A chunk: row r = 2 (m - mi0) + (re|im), k-quad q of chunk starting at k0
  __device__ void a4(int mp, int mi0, int k0, int r, int q, float* x) const {
    const int mi = mi0 + (r >> 1);
    const int m = cs.m0 + mi;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int l = k0 + 4 * q + i;
      float v = 0.f;
      if (l < Lb && mi < cs.Mc && abs(m) <= l) {
        const float f = __ldg(reinterpret_cast<const float*>(flm + (l * l + l + m)) + (r & 1));
        v = dq(Q, Lmax, mp, l, m) * f;
      }
      x[i] = v;
    }
  }
  __device__ void b4(int mp, int n0i, int k0, int c, int q, float* x) const {
    const int ni = n0i + c;
    const int n = cs.n0 + cs.nstep * ni;
    const int N = 2 * Lb - 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int l = k0 + 4 * q + i;
      float v = 0.f;
      if (l < Lb && ni < cs.Nc && abs(n) <= l) v = dq(Q, Lmax, mp, l, n) * __ldg(psi + (size_t)l * N + (n + Lb - 1));
      x[i] = v;
    }
  }
  // 16 accumulator columns [c0, c0+16) of row r; lanes r, r^1 hold re/im of the same m
  __device__ void store16(int mp, int mi0, int n0i, int r, int c0, const float* d) const {
    const int mi = mi0 + (r >> 1);
    const bool odd = r & 1;
    float other[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) other[i] = __shfl_xor_sync(0xffffffffu, d[i], 1);
    if (mi >= cs.Mc) return;
    const int m = cs.m0 + mi;
    const size_t rowbase = ((size_t)mp * cs.Mc + mi) * cs.Nc;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = c0 + (odd ? 8 : 0) + i;
      const int ni = n0i + c;
      if (ni >= cs.Nc) continue;
      const float re = odd ? other[8 + i] : d[i];
      const float im = odd ? d[8 + i] : other[i];
      const int n = cs.n0 + cs.nstep * ni;
      X[rowbase + ni] = mul_ipow(mk<float>(re, im), imod(n - m, 4));
    }
  }
  __device__ void zero16(int mp, int mi0, int n0i, int r, int c0) const {
    float z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0.f;
    store16(mp, mi0, n0i, r, c0, z);
  }
};

struct SynthesisProb {
  const float* Q; int Lmax; const cx<float>* Y; const float* psi; int Lb; ColSet cs; cx<float>* Z;
  // K runs over ni with |n| <= lmax of the l-tile; no work if m' > lmax
  __device__ void tile(int& mp, int& mi0, int& l0, int& kb, int& ke) const {
    mp = blockIdx.z; mi0 = blockIdx.y * (BM / 2); l0 = blockIdx.x * BNC;
    const int lhi = min(l0 + BNC, Lb) - 1;
    if (mp > lhi) { kb = ke = 0; return; }
    const int d = -lhi - cs.n0;
    kb = d <= 0 ? 0 : (d + cs.nstep - 1) / cs.nstep;
    const int dmax = lhi - cs.n0;
    ke = dmax < 0 ? 0 : min(cs.Nc, dmax / cs.nstep + 1);
  }
  __device__ void a4(int mp, int mi0, int k0, int r, int q, float* x) const {
    const int mi = mi0 + (r >> 1);
    const size_t plane = (size_t)cs.Mc * cs.Nc;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ni = k0 + 4 * q + i;
      float v = 0.f;
      if (mi < cs.Mc && ni < cs.Nc) {
        const cx<float> y = Y[(size_t)mp * plane + (size_t)mi * cs.Nc + ni];
        v = (r & 1) ? y.im : y.re;
      }
      x[i] = v;
    }
  }
  __device__ void b4(int mp, int l0, int k0, int c, int q, float* x) const {
    const int l = l0 + c;
    const int N = 2 * Lb - 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ni = k0 + 4 * q + i;
      float v = 0.f;
      if (l < Lb && l >= mp && ni < cs.Nc) {
        const int n = cs.n0 + cs.nstep * ni;
        if (abs(n) <= l) v = dq(Q, Lmax, mp, l, n) * __ldg(psi + (size_t)l * N + (n + Lb - 1));
      }
      x[i] = v;
    }
  }
  __device__ void store16(int mp, int mi0, int l0, int r, int c0, const float* d) const {
    const int mi = mi0 + (r >> 1);
    const bool odd = r & 1;
    float other[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) other[i] = __shfl_xor_sync(0xffffffffu, d[i], 1);
    if (mi >= cs.Mc) return;
    const size_t rowbase = ((size_t)mp * cs.Mc + mi) * Lb;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int l = l0 + c0 + (odd ? 8 : 0) + i;
      if (l >= Lb) continue;
      const float re = odd ? other[8 + i] : d[i];
      const float im = odd ? d[8 + i] : other[i];
      Z[rowbase + l] = mk<float>(re, im);
    }
  }
  __device__ void zero16(int, int, int, int, int) const {}  // tiles without work are never read
};

// f_lm += sum_{m' <= l} Delta^l_{m'm} Z[m'][mi][l] in FP64 (FP64 Delta table).
// Block = 32 (mi) x 32 (l) outputs, 256 threads, m' loop with shared-memory tiles.
__global__ void __launch_bounds__(256) synth_reduce_kernel(const double* __restrict__ Q, int Lmax,
                                                          const cx<float>* __restrict__ Z, int Lb, ColSet cs,
                                                          cx<double>* __restrict__ flm) {
  __shared__ cx<float> Zs[32][33];
  __shared__ double Qs[32][33];  // [l][|m|]
  const int l0 = blockIdx.x * 32, mi0 = blockIdx.y * 32;
  const int lhi = min(l0 + 32, Lb) - 1;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty: 8 rows of mi per pass
  const int mlo = cs.m0 + mi0, mhi = cs.m0 + min(mi0 + 32, cs.Mc) - 1;
  const int amin = (mlo <= 0 && mhi >= 0) ? 0 : min(abs(mlo), abs(mhi));
  if (amin > lhi) return;
  cx<double> acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i] = mk(0.0, 0.0);
  for (int mp = 0; mp <= lhi; ++mp) {
    // Z rows: [mi0 + i][l0 + tx]
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int mi = mi0 + ty + 8 * i, l = l0 + tx;
      Zs[ty + 8 * i][tx] = (mi < cs.Mc && l < Lb) ? Z[((size_t)mp * cs.Mc + mi) * Lb + l] : mk<float>(0, 0);
    }
    // Delta rows: [l0 + i][|m| for the 32 m of the tile]; m = m0 + mi0 + tx
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int l = l0 + ty + 8 * i, m = cs.m0 + mi0 + tx;
      double v = 0.0;
      if (l < Lb && l >= mp && mi0 + tx < cs.Mc && abs(m) <= l) {
        v = Q[((size_t)mp * Lmax + l) * Lmax + abs(m)];
        if (m < 0 && ((l + mp) & 1)) v = -v;
      }
      Qs[ty + 8 * i][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int mloc = ty + 8 * i;  // thread owns (mi0 + mloc, l0 + tx)
      const double d = Qs[tx][mloc];
      const cx<float> z = Zs[mloc][tx];
      acc[i].re += d * (double)z.re;
      acc[i].im += d * (double)z.im;
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int mi = mi0 + ty + 8 * i, l = l0 + tx;
    if (mi >= cs.Mc || l >= Lb) continue;
    const int m = cs.m0 + mi;
    if (abs(m) > l) continue;
    cx<double>& f = flm[l * l + l + m];
    f = f + acc[i];
  }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Host entry points used by crv.cu
// ---------------------------------------------------------------------------
bool tc_analysis(const float* Q32, int Lmax, const cx<float>* flm, const float* psi, int Lb, ColSet cs,
                 cx<float>* X, int* err, cudaStream_t st) {
  tc::AnalysisProb pb{Q32, Lmax, flm, psi, Lb, cs, X};
  dim3 grid((cs.Nc + tc::BNC - 1) / tc::BNC, (cs.Mc + tc::BM / 2 - 1) / (tc::BM / 2), Lb);
  return launch_tc_gemm<tc::AnalysisProb, tc::BNC>(pb, grid, err, st, K_TC_A);
}

bool tc_synthesis(const float* Q32, const double* Q64, int Lmax, const cx<float>* Y, const float* psi, int Lb,
                  ColSet cs, cx<float>* Zscratch, cx<double>* flm, int* err, cudaStream_t st) {
  tc::SynthesisProb pb{Q32, Lmax, Y, psi, Lb, cs, Zscratch};
  dim3 grid((Lb + tc::BNC - 1) / tc::BNC, (cs.Mc + tc::BM / 2 - 1) / (tc::BM / 2), Lb);
  if (!launch_tc_gemm<tc::SynthesisProb, tc::BNC>(pb, grid, err, st, K_TC_S)) return false;
  dim3 g2((Lb + 31) / 32, (cs.Mc + 31) / 32);
  KTimer kt(K_TC_S, st);
  tc::synth_reduce_kernel<<<g2, 256, 0, st>>>(Q64, Lmax, Zscratch, Lb, cs, flm);
  kt.done();
  return launch_ok("synth_reduce_kernel");
}

}  // namespace crv
