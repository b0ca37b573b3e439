// FP64-accurate Delta contractions on the TF32 tensor cores (tcgen05, sm_103a) by
// error-free integer slicing; see tc_ozaki.cuh for the representation and its error.
//
// Analysis, per m' >= 0 (Eq. inverse_Fmnmp, general n, Eq. wav_harmonic_coeff folded in):
//   D[(m, Re|Im)][n] = sum_l A[(m, Re|Im)][l] B[n][l],  A = Delta^l_{m'm} f_lm,
//   B = Delta^l_{m'n} Psi_ln,  X_{m n m'} = i^{n-m} (D_Re + i D_Im);
// synthesis, per m' (Eq. flml, general n, then the n-sum of Eq. wav_synthesis_harmonic):
//   Z[(m, Re|Im)][l] = sum_n A[(m, Re|Im)][n] B[l][n],  A = Y'_{m n m'},  B = Delta^l_{m'n} Psi_ln,
//   f_lm += sum_{m'} Delta^l_{m'm} Z_{m l m'}.
// Both operands are sliced into tables (B once per plan, A per map and per pass over a range
// of m') in the layout of an engine stage, and both come into shared memory by bulk copies.
//
// Engine: persistent, one CTA of 11 warps per SM, tiles taken in order from a global counter.
//   warp 0 (one lane)  schedules tiles into a ring of four slots;
//   warp 1 (one lane)  bulk-copies the A and B chunks of a K step into one of two stages;
//   warp 2 (one lane)  issues, per K step of 8, the OZ_S (OZ_S + 1) / 2 slice products
//                      s + t < OZ_S into five TMEM accumulators of 96 columns (levels 0-3,
//                      and 4 and above together) and commits to the stage's empty barrier;
//   warps 3-10         drain the accumulators (two warps per TMEM lane quarter, half of the
//                      columns each), add them in double-float, scale by the row and
//                      column exponents and store FP64 results (one FP64 add per value).
// Every mbarrier wait is bounded and sets the plan's error flag when it gives up; the other
// roles then stop in turn, copies in flight are waited for and the MMA lane waits for its
// MMAs before TMEM is released.
#include "tc_gemm.cuh"
#include "tc_ozaki.cuh"

namespace crv {
namespace oz {

using tc::bulk_g2s;
using tc::fence_after;
using tc::fence_before;
using tc::mbar_arrive;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_commit;
using tc::mma_drain;
using tc::mma_tf32;
using tc::smem_desc;
using tc::smem_u32;
using tc::tmem_ld16;
using tc::warp_wait;

constexpr int BN = OZ_BROWS;
constexpr int ASL_BYTES = OZ_ASLICE * 4, BSL_BYTES = OZ_BSLICE * 4;  // one slice of a chunk
constexpr int A_BYTES = OZ_ACHUNK * 4, B_BYTES = OZ_BCHUNK * 4;      // all slices of a chunk
constexpr int STAGES = 2, STAGE_BYTES = A_BYTES + B_BYTES, RING = 4;
constexpr int EPI_WARPS = 8;  // two per TMEM lane quarter, each half of the columns
constexpr int THREADS = (3 + EPI_WARPS) * 32;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 512;
constexpr uint32_t TMEM_COLS = 512;
// instruction descriptor: D f32, A/B tf32, K-major A and B, N = 96, M = 128
constexpr uint32_t IDESC =
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(OZ_AROWS >> 4) << 24);
static_assert(OZ_ACCS * BN <= (int)TMEM_COLS, "accumulators fit in TMEM");
static_assert(SMEM_BYTES <= 227 * 1024, "two stages fit in shared memory");
static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "valid MMA N for M = 128");
static_assert((BN / 2) % 16 == 0, "each epilogue warp drains whole 16-column loads");
static_assert(OZ_K == 16 && OZ_AROWS % 8 == 0 && OZ_BROWS % 8 == 0, "stage layout");

// ---------------------------------------------------------------------------
// Slicing
// ---------------------------------------------------------------------------
// Row exponent from the largest |x| as a bit pattern (non-negative doubles order like their
// bits): E with max |x| < 2^E; 0 for a row of zeros and subnormals, which slice to zero.
__device__ __forceinline__ int row_exp(unsigned long long amax_bits) {
  const int ef = (int)(amax_bits >> 52);
  return ef == 0 ? 0 : ef - 1022;
}
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// The OZ_S slices d_k 2^(-bk) of x for the row scale 2^E and b-bit digits, with
// x ~ 2^(E - b + 1) sum_k d_k 2^(-bk), in integer arithmetic: T = round(|x| 2^(OZ_S b - 1 - E))
// from the 53-bit mantissa (|T| <= 2^(OZ_S b - 1)), signed, then balanced base-2^b digits from
// the least significant up, d_k in [-2^(b-1), 2^(b-1)), the top digit taking the rest
// (|d_0| <= 2^(b-1)). One rounding, at 2^(-OZ_S b + 1) of the row scale.
__device__ __forceinline__ void slice(double x, int E, int b, float* d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ef = (int)((u >> 52) & 0x7ff);
  long long T = 0;
  if (ef != 0) {
    const unsigned long long m = (u & 0xfffffffffffffull) | (1ull << 52);  // |x| = m 2^(ef - 1075)
    const int rs = 1076 + E - OZ_S * b - ef;  // >= 54 - OZ_S b (5 for b = 7) because |x| < 2^E
    if (rs < 63) T = (long long)((m + (1ull << (rs - 1))) >> rs);
    if (u >> 63) T = -T;
  }
  const long long mask = (1ll << b) - 1, half = 1ll << (b - 1);
#pragma unroll
  for (int k = OZ_S - 1; k >= 1; --k) {
    long long r = T & mask;
    if (r >= half) r -= mask + 1;
    d[k] = (float)(int)r * __int_as_float((127 - b * k) << 23);
    T = (T - r) >> b;
  }
  d[0] = (float)(int)T;
}

// FP32 -> FP64 by the bit patterns (exact for normal values; zeros and subnormals, which the
// accumulators do not produce above 2^-126 of a result, give 0), so that the epilogue spends
// no FP64 instruction on it.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0) return 0.0;
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                          ((unsigned long long)(ex + 896u) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}
// x 2^e by the exponent field (scalbn when the result leaves the normal range).
__device__ __forceinline__ double scale2(double x, int e) {
  const long long u = __double_as_longlong(x);
  const int ex = (int)((u >> 52) & 0x7ff);
  if (ex == 0) return x;
  const int ne = ex + e;
  if (ne <= 0 || ne >= 2047) return scalbn(x, e);
  return __longlong_as_double(u + ((long long)e << 52));
}

// Four consecutive K values of one row, sliced into the OZ_S slices of the chunk at `chunk`
// (float offset of the row's 16-byte piece: 8-row groups of 128 floats, k-quads 32 floats).
__device__ __forceinline__ void put_slices(float* chunk, int slice_floats, int r, int q, const double* v, int E,
                                           int b) {
  float d[4][OZ_S];
#pragma unroll
  for (int i = 0; i < 4; ++i) slice(v[i], E, b, d[i]);
  float* o = chunk + (r >> 3) * (OZ_K * 8) + q * 32 + (r & 7) * 4;
#pragma unroll
  for (int k = 0; k < OZ_S; ++k)
    *reinterpret_cast<float4*>(o + (size_t)k * slice_floats) = make_float4(d[0][k], d[1][k], d[2][k], d[3][k]);
}

// Fill of a table: block (tile, m' - t.mp0), thread = row of the tile. Two passes over the
// row: its largest magnitude (the row exponent), then the slices. V::at(mp, row, k) is the
// operand value (zero outside the support).
template <int ROWS, class V>
__global__ void __launch_bounds__(128) fill_kernel(V val, OzTab t) {
  const int mpl = blockIdx.y, mp = t.mp0 + mpl, tile = blockIdx.x, r = threadIdx.x;
  if (r >= ROWS) return;
  const size_t idx = (size_t)mpl * t.ntiles + tile;
  const int2 rg = t.range[idx];
  const int row = tile * ROWS + r;
  unsigned long long amax = 0;
  for (int kc = rg.x; kc < rg.x + rg.y; ++kc)
    for (int i = 0; i < OZ_K; ++i) amax = max(amax, abs_bits(val.at(mp, row, kc * OZ_K + i)));
  const int E = row_exp(amax);
  t.e[(size_t)mpl * t.rows + row] = E;
  constexpr int CH = OZ_S * ROWS * OZ_K;
  for (int kc = rg.x; kc < rg.x + rg.y; ++kc) {
    float* chunk = t.v + (size_t)(t.base[idx] - t.c0 + kc) * CH;
#pragma unroll 1
    for (int q = 0; q < OZ_K / 4; ++q) {
      double v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = val.at(mp, row, kc * OZ_K + 4 * q + i);
      put_slices(chunk, ROWS * OZ_K, r, q, v, E, t.bits);
    }
  }
}

// Delta^l_{a,b} for a >= 0 and any b from the FP64 quarter table Q[a][l][|b|].
__device__ __forceinline__ double dq64(const double* __restrict__ Q, int Lmax, int a, int l, int b) {
  const int ab = b < 0 ? -b : b;
  const double v = __ldg(Q + ((size_t)a * Lmax + l) * Lmax + ab);
  return (b < 0 && ((l + a) & 1)) ? -v : v;
}

// Operand values.
struct ValBAnalysis {  // rows n, K = l: Delta^l_{m'n} Psi_ln
  const double* Q; int Lmax; const double* psi; int Lb; ColSet cs;
  __device__ double at(int mp, int ni, int l) const {
    if (ni >= cs.Nc || l >= Lb || l < mp) return 0.0;
    const int n = cs.n0 + cs.nstep * ni;
    if (abs(n) > l) return 0.0;
    return dq64(Q, Lmax, mp, l, n) * psi[(size_t)l * (2 * Lb - 1) + (n + Lb - 1)];
  }
};
struct ValBSynthesis {  // rows l, K = ni: Delta^l_{m'n} Psi_ln
  const double* Q; int Lmax; const double* psi; int Lb; ColSet cs;
  __device__ double at(int mp, int l, int ni) const {
    if (ni >= cs.Nc || l >= Lb || l < mp) return 0.0;
    const int n = cs.n0 + cs.nstep * ni;
    if (abs(n) > l) return 0.0;
    return dq64(Q, Lmax, mp, l, n) * psi[(size_t)l * (2 * Lb - 1) + (n + Lb - 1)];
  }
};
struct ValAAnalysis {  // rows (m, Re|Im), K = l: Delta^l_{m'm} f_lm
  const double* Q; int Lmax; const cx<double>* flm; int Lb; ColSet cs;
  __device__ double at(int mp, int row, int l) const {
    const int mi = row >> 1, m = cs.m0 + mi;
    if (mi >= cs.Mc || l >= Lb || l < mp || abs(m) > l) return 0.0;
    const cx<double> f = flm[l * l + l + m];
    return dq64(Q, Lmax, mp, l, m) * ((row & 1) ? f.im : f.re);
  }
};
struct ValASynthesis {  // rows (m, Re|Im), K = ni: Y'_{m n m'}
  const cx<double>* Y; ColSet cs;
  __device__ double at(int mp, int row, int ni) const {
    const int mi = row >> 1;
    if (mi >= cs.Mc || ni >= cs.Nc) return 0.0;
    const cx<double> y = Y[(size_t)mp * cs.pitch() + cs.col(mi, ni)];
    return (row & 1) ? y.im : y.re;
  }
};

// ---------------------------------------------------------------------------
// Problems: tiles, operand chunks, exponents, epilogues
// ---------------------------------------------------------------------------
struct Tile {
  int mpl, mp, at, bt, c0, nch;  // m' (pass-local, absolute), A tile, B tile, chunk range
};

__device__ __forceinline__ int tile_amin(const ColSet& cs, int at) {
  const int mi0 = at * (OZ_AROWS / 2);
  const int mlo = cs.m0 + mi0, mhi = cs.m0 + min(mi0 + OZ_AROWS / 2, cs.Mc) - 1;
  return (mlo <= 0 && mhi >= 0) ? 0 : min(abs(mlo), abs(mhi));
}

struct AnalysisProb {
  static constexpr bool kZeroEmpty = true;  // X is zero where no l contributes
  OzTab ta, tb; int Lb; ColSet cs; cx<double>* X;
  __device__ void tile(int bx, int by, int bz, Tile& t) const {
    t.mpl = bz; t.mp = ta.mp0 + bz; t.at = by; t.bt = bx;
    const int2 ra = ta.range[(size_t)bz * ta.ntiles + by];
    const int2 rb = tb.range[(size_t)t.mp * tb.ntiles + bx];
    t.c0 = max(ra.x, rb.x);
    const int c1 = min(ra.x + ra.y, rb.x + rb.y);
    t.nch = (ra.y > 0 && rb.y > 0 && c1 > t.c0) ? c1 - t.c0 : 0;
  }
  __device__ const float* a_chunk(const Tile& t, int kc) const {
    return ta.v + (size_t)(ta.base[(size_t)t.mpl * ta.ntiles + t.at] - ta.c0 + kc) * OZ_ACHUNK;
  }
  __device__ const float* b_chunk(const Tile& t, int kc) const {
    return tb.v + (size_t)(tb.base[(size_t)t.mp * tb.ntiles + t.bt] - tb.c0 + kc) * OZ_BCHUNK;
  }
  __device__ int ea(const Tile& t, int r) const { return ta.e[(size_t)t.mpl * ta.rows + t.at * OZ_AROWS + r]; }
  __device__ int eb(const Tile& t, int c) const { return tb.e[(size_t)t.mp * tb.rows + t.bt * OZ_BROWS + c]; }
  // 16 columns [cc, cc + 16) of row r; lanes r, r ^ 1 hold Re and Im of the same m
  __device__ void store16(const Tile& t, int r, int cc, const double* d) const {
    const int mi = t.at * (OZ_AROWS / 2) + (r >> 1);
    const bool odd = r & 1;
    double other[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) other[i] = __shfl_xor_sync(0xffffffffu, d[i], 1);
    if (mi >= cs.Mc) return;
    const int m = cs.m0 + mi;
    cx<double>* plane = X + (size_t)t.mp * cs.pitch();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int ni = t.bt * OZ_BROWS + cc + (odd ? 8 : 0) + i;
      if (ni >= cs.Nc) continue;
      const double re = odd ? other[8 + i] : d[i];
      const double im = odd ? d[8 + i] : other[i];
      const int n = cs.n0 + cs.nstep * ni;
      plane[cs.col(mi, ni)] = mul_ipow(mk(re, im), imod(n - m, 4));
    }
  }
};

struct SynthesisProb {
  static constexpr bool kZeroEmpty = false;  // Z is read only for l >= max(m', |m|)
  OzTab ta, tb; int Lb; ColSet cs; cx<double>* Z;
  // K over ni: the B table's run for (m', l-tile); empty if every |m| of the m-tile exceeds
  // the tile's largest l
  __device__ void tile(int bx, int by, int bz, Tile& t) const {
    t.mpl = bz; t.mp = ta.mp0 + bz; t.at = by; t.bt = bx;
    const int2 rb = tb.range[(size_t)t.mp * tb.ntiles + bx];
    const int lhi = min((bx + 1) * OZ_BROWS, Lb) - 1;
    t.c0 = rb.x;
    t.nch = (rb.y > 0 && tile_amin(cs, by) <= lhi) ? rb.y : 0;
  }
  __device__ const float* a_chunk(const Tile& t, int kc) const {
    return ta.v + (size_t)(ta.base[(size_t)t.mpl * ta.ntiles + t.at] - ta.c0 + kc) * OZ_ACHUNK;
  }
  __device__ const float* b_chunk(const Tile& t, int kc) const {
    return tb.v + (size_t)(tb.base[(size_t)t.mp * tb.ntiles + t.bt] - tb.c0 + kc) * OZ_BCHUNK;
  }
  __device__ int ea(const Tile& t, int r) const { return ta.e[(size_t)t.mpl * ta.rows + t.at * OZ_AROWS + r]; }
  __device__ int eb(const Tile& t, int c) const { return tb.e[(size_t)t.mp * tb.rows + t.bt * OZ_BROWS + c]; }
  __device__ void store16(const Tile& t, int r, int cc, const double* d) const {
    const int mi = t.at * (OZ_AROWS / 2) + (r >> 1);
    const bool odd = r & 1;
    double other[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) other[i] = __shfl_xor_sync(0xffffffffu, d[i], 1);
    if (mi >= cs.Mc) return;
    const size_t rowbase = ((size_t)t.mp * cs.Mc + mi) * Lb;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int l = t.bt * OZ_BROWS + cc + (odd ? 8 : 0) + i;
      if (l >= Lb) continue;
      const double re = odd ? other[8 + i] : d[i];
      const double im = odd ? d[8 + i] : other[i];
      Z[rowbase + l] = mk(re, im);
    }
  }
};

// ---------------------------------------------------------------------------
// The engine
// ---------------------------------------------------------------------------
template <class Prob>
__global__ void __launch_bounds__(THREADS, 1) oz_gemm_kernel(Prob pb, int gx, int gy, int ntiles, int* ctr, int* err) {
  extern __shared__ unsigned char smraw[];
  const uint32_t raw = smem_u32(smraw);
  unsigned char* base = smraw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* tr_full = acc_empty + 1;
  uint64_t* tr_empty = tr_full + RING;
  uint64_t* drain = tr_empty + RING;
  int* tring = reinterpret_cast<int*>(drain + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tring + RING);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, EPI_WARPS);
    for (int i = 0; i < RING; ++i) {
      mbar_init(&tr_full[i], 1);
      mbar_init(&tr_empty[i], 2 + EPI_WARPS);  // copy lane, MMA lane, epilogue warps
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  auto tile_of = [&](int t, Tile& ti) { pb.tile(t % gx, (t / gx) % gy, t / (gx * gy), ti); };

  if (warp == 0) {
    // ---- scheduler: tile indices into the ring; ntiles ends every consumer ----
    if (lane == 0) {
      for (uint32_t j = 0;; ++j) {
        const int sl = j % RING;
        int t = ntiles;
        if (mbar_wait(&tr_empty[sl], ((j / RING) + 1) & 1u, err)) t = min(atomicAdd(ctr, 1), ntiles);
        tring[sl] = t;
        mbar_arrive(&tr_full[sl]);
        if (t >= ntiles) break;
      }
    }
  } else if (warp == 1) {
    // ---- copy lane ----
    if (lane == 0) {
      uint32_t u = 0;
      int last[STAGES];
      for (int i = 0; i < STAGES; ++i) last[i] = -1;
      bool ok = true;
      for (uint32_t j = 0; ok; ++j) {
        const int sl = j % RING;
        if (!mbar_wait(&tr_full[sl], (j / RING) & 1u, err)) break;
        const int t = tring[sl];
        mbar_arrive(&tr_empty[sl]);
        if (t >= ntiles) break;
        Tile ti;
        tile_of(t, ti);
        for (int c = 0; c < ti.nch; ++c, ++u) {
          const int s = u % STAGES;
          if (!mbar_wait(&empty[s], ((u / STAGES) + 1) & 1u, err)) { ok = false; break; }
          unsigned char* st = base + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], (uint32_t)STAGE_BYTES);
          bulk_g2s(st, pb.a_chunk(ti, ti.c0 + c), A_BYTES, &full[s]);
          bulk_g2s(st + A_BYTES, pb.b_chunk(ti, ti.c0 + c), B_BYTES, &full[s]);
          last[s] = (int)u;
        }
      }
      // copies issued and possibly not consumed (an error elsewhere) land before exit
      for (int i = 0; i < STAGES; ++i)
        if (last[i] >= 0) mbar_wait(&full[i], ((uint32_t)last[i] / STAGES) & 1u, err);
    }
  } else if (warp == 2) {
    // ---- MMA lane ----
    if (lane == 0) {
      uint32_t u = 0;
      bool ok = true, issued = false;
      for (uint32_t j = 0; ok; ++j) {
        const int sl = j % RING;
        if (!mbar_wait(&tr_full[sl], (j / RING) & 1u, err)) break;
        const int t = tring[sl];
        mbar_arrive(&tr_empty[sl]);
        if (t >= ntiles) break;
        Tile ti;
        tile_of(t, ti);
        if (!mbar_wait(acc_empty, (j + 1) & 1u, err)) break;
        fence_after();
        uint32_t started = 0;
        for (int c = 0; c < ti.nch; ++c, ++u) {
          const int s = u % STAGES;
          if (!mbar_wait(&full[s], (u / STAGES) & 1u, err)) { ok = false; break; }
          fence_after();
          const uint32_t sa = smem_u32(base + s * STAGE_BYTES), sb = sa + A_BYTES;
#pragma unroll
          for (int ks = 0; ks < OZ_K / 8; ++ks) {
#pragma unroll
            for (int lv = 0; lv < OZ_S; ++lv) {
              const int g = lv < OZ_EXACT_LEVELS ? lv : OZ_EXACT_LEVELS;
#pragma unroll
              for (int a = 0; a <= lv; ++a) {
                const uint64_t da = smem_desc(sa + a * ASL_BYTES + ks * 256);
                const uint64_t db = smem_desc(sb + (lv - a) * BSL_BYTES + ks * 256);
                mma_tf32(tmem + (uint32_t)(g * BN), da, db, IDESC, (started >> g) & 1u);
                started |= 1u << g;
              }
            }
          }
          issued = true;
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        if (ti.nch > 0) mma_commit(acc_full);
        else mbar_arrive(acc_full);
      }
      if (issued) mma_drain(drain, err);
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns of half (w - 3) / 4 ----
    const int lq = warp & 3, r = lq * 32 + lane;
    const int cbeg = ((warp - 3) / 4) * (BN / 2), cend = cbeg + BN / 2;
    for (uint32_t j = 0;; ++j) {
      const int sl = j % RING;
      if (!warp_wait(&tr_full[sl], (j / RING) & 1u, err)) break;
      const int t = tring[sl];
      __syncwarp();
      if (lane == 0) mbar_arrive(&tr_empty[sl]);
      if (t >= ntiles) break;
      Tile ti;
      tile_of(t, ti);
      if (!warp_wait(acc_full, j & 1u, err)) break;
      fence_after();
      const int er = ti.nch > 0 ? pb.ea(ti, r) : 0;
      const int eoff = 2 * (pb.ta.bits - 1);  // x = 2^(E - b + 1) sum_k d_k 2^(-bk) for both operands
      for (int cc = cbeg; cc < cend; cc += 16) {
        double v[16];
        if (ti.nch > 0) {
          float a[OZ_ACCS][16];
#pragma unroll
          for (int g = 0; g < OZ_ACCS; ++g)
            tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(g * BN + cc), a[g]);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            // levels 0 and 1 (and 2) exactly as a double-float (h, lo), the rest added to lo
            float h = a[0][i] + a[1][i];
            float bb = h - a[0][i];
            float lo = (a[0][i] - (h - bb)) + (a[1][i] - bb);
            const float h2 = h + a[2][i];
            bb = h2 - h;
            lo += (h - (h2 - bb)) + (a[2][i] - bb);
            h = h2;
#pragma unroll
            for (int g = 3; g < OZ_ACCS; ++g) lo += a[g][i];
            v[i] = scale2(f2d(h) + f2d(lo), er + pb.eb(ti, cc + i) - eoff);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.0;
        }
        if (ti.nch > 0 || Prob::kZeroEmpty) pb.store16(ti, r, cc, v);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
  }
  __syncwarp();
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// f_lm += sum_{m' <= l} Delta^l_{m'm} Z[m'][mi][l] in FP64, one thread per (l, m), threads
// of a block along l; Delta^l_{m'm} read as Delta^l_{|m| m'} (contiguous in m'):
//   m >= 0: Delta^l_{m'm} = (-1)^{m'+m} Q[m][l][m'],   m < 0: (-1)^{l+|m|} Q[|m|][l][m'].
__global__ void __launch_bounds__(256) reduce_kernel(const double* __restrict__ Q, int Lmax,
                                                    const cx<double>* __restrict__ Z, int Lb, ColSet cs,
                                                    cx<double>* __restrict__ flm) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x, mi = blockIdx.y;
  const int m = cs.m0 + mi, am = m < 0 ? -m : m;
  if (l >= Lb || am > l) return;
  const double* __restrict__ q = Q + ((size_t)am * Lmax + l) * Lmax;
  const cx<double>* __restrict__ z = Z + (size_t)mi * Lb + l;
  const size_t zs = (size_t)cs.Mc * Lb;
  const double so = m >= 0 ? -1.0 : 1.0;
  cx<double> acc = mk(0.0, 0.0);
  for (int mp = 0; mp <= l; ++mp) {
    const double d = (mp & 1) ? so * __ldg(q + mp) : __ldg(q + mp);
    const cx<double> v = z[(size_t)mp * zs];
    acc.re = fma(d, v.re, acc.re);
    acc.im = fma(d, v.im, acc.im);
  }
  const bool neg = m >= 0 ? (am & 1) : ((l + am) & 1);
  cx<double>& f = flm[l * l + l + m];
  f = neg ? f - acc : f + acc;
}

}  // namespace oz

// ---------------------------------------------------------------------------
// Host
// ---------------------------------------------------------------------------
void oz_ranges_b_analysis(int Lb, const ColSet& cs, std::vector<int2>& range, int& ntiles) {
  ntiles = (cs.Nc + OZ_BROWS - 1) / OZ_BROWS;
  const int nchunk = (Lb + OZ_K - 1) / OZ_K;
  range.assign((size_t)Lb * ntiles, make_int2(0, 0));
  for (int mp = 0; mp < Lb; ++mp)
    for (int t = 0; t < ntiles; ++t) {
      const int nlo = cs.n0 + cs.nstep * (t * OZ_BROWS);
      const int nhi = cs.n0 + cs.nstep * (std::min((t + 1) * OZ_BROWS, cs.Nc) - 1);
      const int bmin = (nlo <= 0 && nhi >= 0) ? 0 : std::min(std::abs(nlo), std::abs(nhi));
      const int kb = std::max(mp, bmin);
      if (kb >= Lb) continue;
      range[(size_t)mp * ntiles + t] = make_int2(kb / OZ_K, nchunk - kb / OZ_K);
    }
}

void oz_ranges_b_synthesis(int Lb, const ColSet& cs, std::vector<int2>& range, int& ntiles) {
  ntiles = (Lb + OZ_BROWS - 1) / OZ_BROWS;
  range.assign((size_t)Lb * ntiles, make_int2(0, 0));
  for (int mp = 0; mp < Lb; ++mp)
    for (int t = 0; t < ntiles; ++t) {
      const int lhi = std::min((t + 1) * OZ_BROWS, Lb) - 1;
      if (mp > lhi) continue;
      const int d = -lhi - cs.n0, dmax = lhi - cs.n0;  // ni with |n| <= lhi: [kb, ke)
      const int kb = d <= 0 ? 0 : (d + cs.nstep - 1) / cs.nstep;
      const int ke = dmax < 0 ? 0 : std::min(cs.Nc, dmax / cs.nstep + 1);
      if (ke <= kb) continue;
      const int c0 = kb / OZ_K, c1 = (ke + OZ_K - 1) / OZ_K;
      range[(size_t)mp * ntiles + t] = make_int2(c0, c1 - c0);
    }
}

void oz_ranges_a_analysis(int Lb, const ColSet& cs, std::vector<int2>& range, int& ntiles) {
  ntiles = (cs.Mc + OZ_AROWS / 2 - 1) / (OZ_AROWS / 2);
  const int nchunk = (Lb + OZ_K - 1) / OZ_K;
  range.assign((size_t)Lb * ntiles, make_int2(0, 0));
  for (int mp = 0; mp < Lb; ++mp)
    for (int t = 0; t < ntiles; ++t) {
      const int mlo = cs.m0 + t * (OZ_AROWS / 2), mhi = cs.m0 + std::min((t + 1) * (OZ_AROWS / 2), cs.Mc) - 1;
      const int amin = (mlo <= 0 && mhi >= 0) ? 0 : std::min(std::abs(mlo), std::abs(mhi));
      const int kb = std::max(mp, amin);
      if (kb >= Lb) continue;
      range[(size_t)mp * ntiles + t] = make_int2(kb / OZ_K, nchunk - kb / OZ_K);
    }
}

void oz_ranges_a_synthesis(int Lb, const ColSet& cs, std::vector<int2>& range, int& ntiles) {
  ntiles = (cs.Mc + OZ_AROWS / 2 - 1) / (OZ_AROWS / 2);
  const int nchunk = (cs.Nc + OZ_K - 1) / OZ_K;
  range.assign((size_t)Lb * ntiles, make_int2(0, nchunk));
}

bool oz_fill_b_analysis(const double* Q, int Lmax, const double* psi, int Lb, ColSet cs, OzTab t, cudaStream_t st) {
  KTimer kt(K_MISC, st);
  oz::fill_kernel<OZ_BROWS, oz::ValBAnalysis><<<dim3(t.ntiles, t.mp1 - t.mp0), 128, 0, st>>>(
      oz::ValBAnalysis{Q, Lmax, psi, Lb, cs}, t);
  kt.done();
  return launch_ok("oz fill_kernel (B, analysis)");
}

bool oz_fill_b_synthesis(const double* Q, int Lmax, const double* psi, int Lb, ColSet cs, OzTab t, cudaStream_t st) {
  KTimer kt(K_MISC, st);
  oz::fill_kernel<OZ_BROWS, oz::ValBSynthesis><<<dim3(t.ntiles, t.mp1 - t.mp0), 128, 0, st>>>(
      oz::ValBSynthesis{Q, Lmax, psi, Lb, cs}, t);
  kt.done();
  return launch_ok("oz fill_kernel (B, synthesis)");
}

// Persistent launch over gx x gy x gz tiles (one CTA per SM at most); ctr is zeroed here.
template <class Prob>
static bool launch_oz(const Prob& pb, int gx, int gy, int gz, int* ctr, int* err, cudaStream_t st, int kind) {
  if (!func_attr_once((const void*)oz::oz_gemm_kernel<Prob>, oz::SMEM_BYTES)) return false;
  const long long nt = (long long)gx * gy * gz;
  if (nt <= 0) return true;
  if (nt > 0x7fffffffLL) return false;
  const int ctas = (int)std::min<long long>(nt, device_sms());
  if (cudaMemsetAsync(ctr, 0, sizeof(int), st) != cudaSuccess) return false;
  KTimer kt(kind, st);
  oz::oz_gemm_kernel<Prob><<<ctas, oz::THREADS, oz::SMEM_BYTES, st>>>(pb, gx, gy, (int)nt, ctr, err);
  kt.done();
  return launch_ok(kind_name(kind));
}

bool oz_analysis(const double* Q, int Lmax, const cx<double>* flm, OzTab ta, OzTab tb, int Lb, ColSet cs,
                 cx<double>* X, int* err, int* ctr, cudaStream_t st) {
  const int gz = ta.mp1 - ta.mp0;
  if (gz <= 0) return true;
  {
    KTimer kt(K_OZ_A, st);
    oz::fill_kernel<OZ_AROWS, oz::ValAAnalysis><<<dim3(ta.ntiles, gz), 128, 0, st>>>(
        oz::ValAAnalysis{Q, Lmax, flm, Lb, cs}, ta);
    kt.done();
    if (!launch_ok("oz fill_kernel (A, analysis)")) return false;
  }
  oz::AnalysisProb pb{ta, tb, Lb, cs, X};
  return launch_oz(pb, tb.ntiles, ta.ntiles, gz, ctr, err, st, K_OZ_A);
}

bool oz_synthesis_products(const cx<double>* Y, OzTab ta, OzTab tb, int Lb, ColSet cs, cx<double>* Z, int* err,
                           int* ctr, cudaStream_t st) {
  const int gz = ta.mp1 - ta.mp0;
  if (gz <= 0) return true;
  {
    KTimer kt(K_OZ_S, st);
    oz::fill_kernel<OZ_AROWS, oz::ValASynthesis><<<dim3(ta.ntiles, gz), 128, 0, st>>>(oz::ValASynthesis{Y, cs}, ta);
    kt.done();
    if (!launch_ok("oz fill_kernel (A, synthesis)")) return false;
  }
  oz::SynthesisProb pb{ta, tb, Lb, cs, Z};
  return launch_oz(pb, tb.ntiles, ta.ntiles, gz, ctr, err, st, K_OZ_S);
}

bool oz_synthesis_reduce(const double* Q, int Lmax, const cx<double>* Z, int Lb, ColSet cs, cx<double>* flm,
                         cudaStream_t st) {
  KTimer kt(K_OZ_S, st);
  oz::reduce_kernel<<<dim3((Lb + 255) / 256, cs.Mc), 256, 0, st>>>(Q, Lmax, Z, Lb, cs, flm);
  kt.done();
  return launch_ok("oz reduce_kernel");
}

}  // namespace crv
