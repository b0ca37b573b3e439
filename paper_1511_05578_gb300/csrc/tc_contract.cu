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
#include <cstdint>

#include "transforms.cuh"

namespace crv {
namespace tc {

constexpr int BM = 128, BN = 256, BK = 32, STAGES = 2, NT = 512;
constexpr int A_BYTES = BM * BK * 4;             // 16 KB per A tile (hi or lo)
constexpr int B_BYTES = BN * BK * 4;             // 32 KB per B tile (hi or lo)
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 2048;
constexpr long kWaitLimit = 1L << 22;            // bounded spin on mbarriers

// instruction descriptor: D f32, A/B tf32, K-major A and B, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of the 16-byte chunk (row r, k-quad q) in a [rows x 32] tf32 tile:
// core matrix (8 rows x 16 B) at (r/8, q); K-adjacent core matrices 128 B apart,
// 8-row groups 1024 B apart.
__device__ __forceinline__ uint32_t chunk_off(int r, int q) { return (uint32_t)((r >> 3) * 1024 + q * 128 + (r & 7) * 16); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;   // leading byte offset: next core matrix along K
  d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
  return d;                           // base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) atomicExch(err, 1);
  return false;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Store four FP32 values as tf32 hi and lo into the (r, q) chunk of the hi and lo tiles.
__device__ __forceinline__ void put4(unsigned char* hi_tile, unsigned char* lo_tile, int r, int q, const float* x) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = tf32_rna(x[i]);
    l[i] = tf32_rna(x[i] - __uint_as_float(h[i]));
  }
  const uint32_t off = chunk_off(r, q);
  *reinterpret_cast<uint4*>(hi_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ float dq(const float* __restrict__ Q, int Lmax, int a, int l, int b) {
  const int ab = b < 0 ? -b : b;
  float v = __ldg(Q + ((size_t)a * Lmax + l) * Lmax + ab);
  return (b < 0 && ((l + a) & 1)) ? -v : v;
}

// ---------------------------------------------------------------------------
// Problems: operand builders, K ranges and epilogues
// ---------------------------------------------------------------------------
struct AnalysisProb {
  const float* Q; int Lmax; const cx<float>* flm; const float* psi; int Lb; ColSet cs; cx<float>* X;
  __device__ void tile(int& mp, int& mi0, int& n0i, int& kb, int& ke) const {
    mp = blockIdx.z; mi0 = blockIdx.y * (BM / 2); n0i = blockIdx.x * BN;
    const int mlo = cs.m0 + mi0, mhi = cs.m0 + min(mi0 + BM / 2, cs.Mc) - 1;
    const int nlo = cs.n0 + cs.nstep * n0i, nhi = cs.n0 + cs.nstep * (min(n0i + BN, cs.Nc) - 1);
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
    mp = blockIdx.z; mi0 = blockIdx.y * (BM / 2); l0 = blockIdx.x * BN;
    const int lhi = min(l0 + BN, Lb) - 1;
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

// ---------------------------------------------------------------------------
// The GEMM kernel: one 128 x 128 output tile per CTA.
// ---------------------------------------------------------------------------
template <class Prob>
__global__ void __launch_bounds__(NT, 1) tc_gemm_kernel(Prob pb, int* err) {
  extern __shared__ unsigned char smraw[];
  const uint32_t raw = smem_u32(smraw);
  unsigned char* base = smraw + (((raw + 1023u) & ~1023u) - raw);  // 1024-byte aligned stage buffers
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + STAGES);
  const int tid = threadIdx.x, warp = tid >> 5;

  int mp, r0, c0g, kb, ke;
  pb.tile(mp, r0, c0g, kb, ke);
  const int nchunks = (ke > kb) ? (ke - kb + BK - 1) / BK : 0;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  for (int c = 0; c < nchunks; ++c) {
    const int s = c % STAGES;
    if (c >= STAGES) ok = mbar_wait(&bars[s], (uint32_t)((c / STAGES) - 1) & 1u, err) && ok;
    unsigned char* st = base + s * STAGE_BYTES;
    const int k0 = kb + c * BK;
    // A: 128 rows x 8 k-quads, B: 256 rows x 8 k-quads; 2 + 4 chunks per thread.
    // All loads of a thread are issued before any split/store (latency hiding).
    {
      constexpr int NA = BM * (BK / 4) / NT, NB = BN * (BK / 4) / NT;
      float xa[NA][4], xb[NB][4];
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const int it = tid + i * NT;
        pb.a4(mp, r0, k0, it % BM, it / BM, xa[i]);
      }
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int it = tid + i * NT;
        pb.b4(mp, c0g, k0, it % BN, it / BN, xb[i]);
      }
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const int it = tid + i * NT;
        put4(st, st + A_BYTES, it % BM, it / BM, xa[i]);
      }
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int it = tid + i * NT;
        put4(st + 2 * A_BYTES, st + 2 * A_BYTES + B_BYTES, it % BN, it / BN, xb[i]);
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0 && ok) {
      fence_after();
      const uint32_t sa = smem_u32(st);
#pragma unroll
      for (int ks = 0; ks < BK / 8; ++ks) {
        const uint32_t koff = ks * 256;  // two core matrices (8 tf32) per K-step
        const uint64_t ahi = smem_desc(sa + koff), alo = smem_desc(sa + A_BYTES + koff);
        const uint64_t bhi = smem_desc(sa + 2 * A_BYTES + koff), blo = smem_desc(sa + 2 * A_BYTES + B_BYTES + koff);
        const uint32_t first = (c == 0 && ks == 0) ? 0u : 1u;
        mma_tf32(tmem, alo, bhi, first);
        mma_tf32(tmem, ahi, blo, 1u);
        mma_tf32(tmem, ahi, bhi, 1u);
      }
      mma_commit(&bars[s]);
    }
  }
  if (nchunks > 0) {
    const int last = nchunks - 1;
    ok = mbar_wait(&bars[last % STAGES], (uint32_t)(last / STAGES) & 1u, err) && ok;
  }
  fence_after();
  if (warp < 4) {
    const int r = warp * 32 + (tid & 31);
    for (int cc = 0; cc < BN; cc += 16) {
      if (nchunks > 0 && ok) {
        float d[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, d);
        pb.store16(mp, r0, c0g, r, cc, d);
      } else {
        pb.zero16(mp, r0, c0g, r, cc);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

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
size_t tc_scratch_bytes(int, int, int) { return 0; }

template <class Prob>
static bool launch_gemm(const Prob& pb, dim3 grid, int* err, cudaStream_t st, int kind) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tc::tc_gemm_kernel<Prob>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc::SMEM_BYTES) != cudaSuccess)
      return false;
    attr = true;
  }
  KTimer kt(kind, st);
  tc::tc_gemm_kernel<Prob><<<grid, tc::NT, tc::SMEM_BYTES, st>>>(pb, err);
  kt.done();
  return launch_ok(kind_name(kind));
}

bool tc_analysis(const float* Q32, int Lmax, const cx<float>* flm, const float* psi, int Lb, ColSet cs,
                 cx<float>* X, int* err, cudaStream_t st) {
  tc::AnalysisProb pb{Q32, Lmax, flm, psi, Lb, cs, X};
  dim3 grid((cs.Nc + tc::BN - 1) / tc::BN, (cs.Mc + tc::BM / 2 - 1) / (tc::BM / 2), Lb);
  return launch_gemm(pb, grid, err, st, K_TC_A);
}

bool tc_synthesis(const float* Q32, const double* Q64, int Lmax, const cx<float>* Y, const float* psi, int Lb,
                  ColSet cs, cx<float>* Zscratch, cx<double>* flm, int* err, cudaStream_t st) {
  tc::SynthesisProb pb{Q32, Lmax, Y, psi, Lb, cs, Zscratch};
  dim3 grid((Lb + tc::BN - 1) / tc::BN, (cs.Mc + tc::BM / 2 - 1) / (tc::BM / 2), Lb);
  if (!launch_gemm(pb, grid, err, st, K_TC_S)) return false;
  dim3 g2((Lb + 31) / 32, (cs.Mc + 31) / 32);
  KTimer kt(K_TC_S, st);
  tc::synth_reduce_kernel<<<g2, 256, 0, st>>>(Q64, Lmax, Zscratch, Lb, cs, flm);
  kt.done();
  return launch_ok("synth_reduce_kernel");
}

}  // namespace crv
