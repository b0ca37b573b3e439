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
// product). The B operand (Delta Psi, independent of the signal) comes from tables built
// once per plan, already split and in the layout of an engine stage, by bulk copies; the A
// operand is built on the fly. See tc_gemm.cuh for the pipeline.
#include "tc_contract.cuh"
#include "tc_gemm.cuh"

namespace crv {
namespace tc {

constexpr int BNC = 256;  // accumulator width of the contraction tiles
static_assert(BNC == TC_TILE_ROWS, "table tiles are accumulator tiles");

// ---------------------------------------------------------------------------
// Problems: operand builders, K ranges and epilogues
// ---------------------------------------------------------------------------
// Hi and lo B tiles of the K step starting at k0 (a multiple of BK) for (m', tile).
__device__ __forceinline__ void tab_tiles(const TcTab& tb, int mp, int tile, int k0, const void*& hi,
                                          const void*& lo) {
  static_assert(TC_CHUNK_K == BK, "one table chunk per engine stage");
  const size_t off = (size_t)(tb.base[mp * tb.ntiles + tile] + k0 / TC_CHUNK_K) * TC_CHUNK_FLOATS;
  hi = tb.hi + off;
  lo = tb.lo + off;
}

struct AnalysisProb {
  static constexpr bool kBulkB = true;
  const float* Q; int Lmax; const cx<float>* flm; TcTab tb; int Lb; ColSet cs; cx<float>* X;
  bool split = false;  // hi*hi apart from the corrections (scales with long l runs)
  // K chunks: the table's run for (m', n-tile), skipping chunks below min |m| of the m-tile
  __device__ void tile(int bx, int by, int bz, int& mp, int& mi0, int& n0i, int& kb, int& ke) const {
    mp = bz; mi0 = by * (BM / 2); n0i = bx * BNC;
    const int2 ch = tc_analysis_tile_chunks(tb.range[mp * tb.ntiles + bx], tc_tile_amin(cs, mi0, BM / 2));
    kb = ch.x * TC_CHUNK_K;
    ke = ch.y * TC_CHUNK_K;
  }
  // A chunk: row r = 2 (m - mi0) + (re|im), k-quad q of chunk starting at k0
  __device__ void a4(int mp, int mi0, int k0, int r, int q, float* x) const {
    const int mi = mi0 + (r >> 1);
    const int m = cs.m0 + mi;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int l = k0 + 4 * q + i;
      float v = 0.f;
      if (l < Lb && l >= mp && mi < cs.Mc && abs(m) <= l) {
        const float f = __ldg(reinterpret_cast<const float*>(flm + (l * l + l + m)) + (r & 1));
        v = dq(Q, Lmax, mp, l, m) * f;
      }
      x[i] = v;
    }
  }
  __device__ void b_tiles(int mp, int n0i, int k0, const void*& hi, const void*& lo) const {
    tab_tiles(tb, mp, n0i / BNC, k0, hi, lo);
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
    cx<float>* plane = X + (size_t)mp * cs.pitch();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = c0 + (odd ? 8 : 0) + i;
      const int ni = n0i + c;
      if (ni >= cs.Nc) continue;
      const float re = odd ? other[8 + i] : d[i];
      const float im = odd ? d[8 + i] : other[i];
      const int n = cs.n0 + cs.nstep * ni;
      plane[cs.col(mi, ni)] = mul_ipow(mk<float>(re, im), imod(n - m, 4));
    }
  }
  __device__ void zero16(int mp, int mi0, int n0i, int r, int c0) const {
    float z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0.f;
    store16(mp, mi0, n0i, r, c0, z);
  }
};

// Analysis with the A operand from the per-map tables (persistent engine).
struct AnalysisProbA : AnalysisProb {
  static constexpr bool kBulkA = true;
  TcATab ta;
  __device__ void a_tiles(int mp, int mi0, int k0, const void*& hi, const void*& lo) const {
    const size_t off =
        (size_t)(ta.base[mp * ta.nmt + mi0 / (BM / 2)] + k0 / TC_CHUNK_K) * TC_ACHUNK_FLOATS;
    hi = ta.hi + off;
    lo = ta.lo + off;
  }
};

struct SynthesisProb {
  static constexpr bool kBulkB = true;
  static constexpr bool kPairLoads = true;
  const cx<float>* Y; TcTab tb; int Lb; ColSet cs; cx<float>* Z;
  // K chunks over ni: the table's run for (m', l-tile); empty if m' > max l of the tile, or
  // if every |m| of the m-tile exceeds it (Z_{m l m'} is read only for l >= |m|)
  __device__ void tile(int bx, int by, int bz, int& mp, int& mi0, int& l0, int& kb, int& ke) const {
    mp = bz; mi0 = by * (BM / 2); l0 = bx * BNC;
    const int2 rg = tb.range[mp * tb.ntiles + bx];
    const int amin = tc_tile_amin(cs, mi0, BM / 2);
    const int lhi = min(l0 + BNC, Lb) - 1;
    kb = rg.x * TC_CHUNK_K;
    ke = amin > lhi ? kb : (rg.x + rg.y) * TC_CHUNK_K;
  }
  // Pair loads: lane r & 3 = j of the four rows r = 4p .. 4p+3 (m = mi0 + 2p and its pair
  // partner, Re and Im) takes the 16 bytes of both columns at ni = k0 + 4q + j, i.e. the four
  // rows at one K; the engine transposes the group (rows out of range are zeroed by a_rows).
  __device__ void a4(int mp, int mi0, int k0, int r, int q, float* x) const {
    const int mi = mi0 + ((r >> 2) << 1);  // first m of the pair (mi0 is even)
    const int ni = k0 + 4 * q + (r & 3);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mi < cs.Mc && ni < cs.Nc)  // the partner column of an odd Mc is in the plane's pitch
      v = *reinterpret_cast<const float4*>(Y + (size_t)mp * cs.pitch() + cs.col(mi, ni));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
  __device__ void a_rows(int mi0, int r, float* x) const {
    if (mi0 + (r >> 1) >= cs.Mc) x[0] = x[1] = x[2] = x[3] = 0.f;
  }
  __device__ void b_tiles(int mp, int l0, int k0, const void*& hi, const void*& lo) const {
    tab_tiles(tb, mp, l0 / BNC, k0, hi, lo);
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

// f_lm += sum_{m' <= l} Delta^l_{m'm} Z[m'][mi][l] (Eq. flml's sum over m'), one thread per
// (l, m) with l >= lmin (below the kernel's support Z is zero and its tiles are not
// computed), threads of a block along l (Z reads coalesced). Delta^l_{m'm} is read as
// Delta^l_{|m| m'} from the FP32 table, contiguous in m' for each thread: with
// Delta^l_{m'm} = (-1)^{m'-m} Delta^l_{mm'} and Delta^l_{m',-n} = (-1)^{l+m'} Delta^l_{m'n},
//   m >= 0: Delta^l_{m'm} = (-1)^{m'+m} Q[m][l][m'],   m < 0: (-1)^{l+|m|} Q[|m|][l][m'].
// Products and partial sums in FP32, flushed into an FP64 accumulator every 32 terms;
// f_lm accumulates in FP64.
__global__ void __launch_bounds__(256) synth_reduce_kernel(const float* __restrict__ Q32, int Lmax,
                                                          const cx<float>* __restrict__ Z, int Lb, int lmin,
                                                          ColSet cs, cx<double>* __restrict__ flm) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x, mi = blockIdx.y;
  const int m = cs.m0 + mi, am = m < 0 ? -m : m;
  if (l >= Lb || l < lmin || am > l) return;
  const float* __restrict__ q = Q32 + ((size_t)am * Lmax + l) * Lmax;  // q[m'] = Delta^l_{|m| m'}
  const cx<float>* __restrict__ z = Z + (size_t)mi * Lb + l;           // z[m' * Mc * Lb]
  const size_t zs = (size_t)cs.Mc * Lb;
  cx<double> acc = mk(0.0, 0.0);  // sum over even m' minus (m >= 0) / plus (m < 0) odd m'
  const float so = m >= 0 ? -1.f : 1.f;
  for (int m0 = 0; m0 <= l; m0 += 32) {
    float er = 0.f, ei = 0.f;
    const int mend = min(m0 + 32, l + 1);
    for (int mp = m0; mp < mend; ++mp) {
      const float d = (mp & 1) ? so * __ldg(q + mp) : __ldg(q + mp);
      const cx<float> v = z[(size_t)mp * zs];
      er = fmaf(d, v.re, er);
      ei = fmaf(d, v.im, ei);
    }
    acc.re += (double)er;
    acc.im += (double)ei;
  }
  const bool neg = m >= 0 ? (am & 1) : ((l + am) & 1);
  cx<double>& f = flm[l * l + l + m];
  f = neg ? f - acc : f + acc;
}

// Self-test of the error path of the bounded waits: one thread waits on an mbarrier that
// nothing arrives at, with a limit of `limit` polls; the wait gives up and sets *err. No
// other thread, copy or MMA is involved, so nothing is left in flight.
__global__ void bounded_wait_probe_kernel(int* err, long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_wait(&bar, 0u, err, limit);
}

// Four values as TF32 hi = rna(x) and lo = rna(x - hi) at float offset o of the two tables.
__device__ __forceinline__ void put_split4(float* hi, float* lo, size_t o, const float* x) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = tf32_rna(x[i]);
    l[i] = tf32_rna(x[i] - __uint_as_float(h[i]));
  }
  *reinterpret_cast<uint4*>(hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Table fills: block (tile, m'), thread = row of the 256-row chunks.
__global__ void __launch_bounds__(256) fill_analysis_table_kernel(const float* __restrict__ Q, int Lmax,
                                                                 const float* __restrict__ psi, int Lb, ColSet cs,
                                                                 TcTab t, float* __restrict__ hi,
                                                                 float* __restrict__ lo) {
  const int mp = blockIdx.y, tile = blockIdx.x, r = threadIdx.x;
  const int2 rg = t.range[mp * t.ntiles + tile];
  const long long base = t.base[mp * t.ntiles + tile];
  const int ni = tile * TC_TILE_ROWS + r, n = cs.n0 + cs.nstep * ni, N = 2 * Lb - 1;
  for (int kc = rg.x; kc < rg.x + rg.y; ++kc) {
    const size_t chunk = (size_t)(base + kc) * TC_CHUNK_FLOATS;
#pragma unroll 1
    for (int q = 0; q < TC_CHUNK_K / 4; ++q) {
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int l = kc * TC_CHUNK_K + 4 * q + i;
        v[i] = (ni < cs.Nc && l < Lb && l >= mp && abs(n) <= l)
                   ? dq(Q, Lmax, mp, l, n) * psi[(size_t)l * N + (n + Lb - 1)]
                   : 0.f;
      }
      put_split4(hi, lo, chunk + (r >> 3) * (TC_CHUNK_K * 8) + q * 32 + (r & 7) * 4, v);
    }
  }
}
__global__ void __launch_bounds__(256) fill_synthesis_table_kernel(const float* __restrict__ Q, int Lmax,
                                                                  const float* __restrict__ psi, int Lb, ColSet cs,
                                                                  TcTab t, float* __restrict__ hi,
                                                                 float* __restrict__ lo) {
  const int mp = blockIdx.y, tile = blockIdx.x, r = threadIdx.x;
  const int2 rg = t.range[mp * t.ntiles + tile];
  const long long base = t.base[mp * t.ntiles + tile];
  const int l = tile * TC_TILE_ROWS + r, N = 2 * Lb - 1;
  for (int kc = rg.x; kc < rg.x + rg.y; ++kc) {
    const size_t chunk = (size_t)(base + kc) * TC_CHUNK_FLOATS;
#pragma unroll 1
    for (int q = 0; q < TC_CHUNK_K / 4; ++q) {
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int ni = kc * TC_CHUNK_K + 4 * q + i, n = cs.n0 + cs.nstep * ni;
        v[i] = (l < Lb && l >= mp && ni < cs.Nc && abs(n) <= l)
                   ? dq(Q, Lmax, mp, l, n) * psi[(size_t)l * N + (n + Lb - 1)]
                   : 0.f;
      }
      put_split4(hi, lo, chunk + (r >> 3) * (TC_CHUNK_K * 8) + q * 32 + (r & 7) * 4, v);
    }
  }
}

// Per-map A tables of the analysis: block (m-tile, m'), thread = row r = 2 (m - mi0) + Re|Im.
__global__ void __launch_bounds__(TC_A_ROWS) fill_analysis_a_kernel(const float* __restrict__ Q, int Lmax,
                                                                     const cx<float>* __restrict__ flm, int Lb,
                                                                     ColSet cs, TcATab t) {
  const int mp = blockIdx.y, mt = blockIdx.x, r = threadIdx.x;
  const int2 rg = t.range[mp * t.nmt + mt];
  const long long base = t.base[mp * t.nmt + mt];
  const int mi = mt * (TC_A_ROWS / 2) + (r >> 1), m = cs.m0 + mi, am = m < 0 ? -m : m;
  const bool row_ok = mi < cs.Mc;
  for (int kc = rg.x; kc < rg.x + rg.y; ++kc) {
    const size_t chunk = (size_t)(base + kc) * TC_ACHUNK_FLOATS;
#pragma unroll 1
    for (int q = 0; q < TC_CHUNK_K / 4; ++q) {
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int l = kc * TC_CHUNK_K + 4 * q + i;
        float x = 0.f;
        if (row_ok && l < Lb && l >= mp && am <= l) {
          const float f = __ldg(reinterpret_cast<const float*>(flm + (l * l + l + m)) + (r & 1));
          x = dq(Q, Lmax, mp, l, m) * f;
        }
        v[i] = x;
      }
      put_split4(t.hi, t.lo, chunk + (r >> 3) * (TC_CHUNK_K * 8) + q * 32 + (r & 7) * 4, v);
    }
  }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Host entry points used by crv.cu
// ---------------------------------------------------------------------------
void tc_analysis_ranges(int Lb, int lmin, const ColSet& cs, std::vector<int2>& range, int& ntiles) {
  ntiles = (cs.Nc + TC_TILE_ROWS - 1) / TC_TILE_ROWS;
  const int nchunk = (Lb + TC_CHUNK_K - 1) / TC_CHUNK_K;
  range.assign((size_t)Lb * ntiles, make_int2(0, 0));
  for (int mp = 0; mp < Lb; ++mp)
    for (int t = 0; t < ntiles; ++t) {
      const int nlo = cs.n0 + cs.nstep * (t * TC_TILE_ROWS);
      const int nhi = cs.n0 + cs.nstep * (std::min((t + 1) * TC_TILE_ROWS, cs.Nc) - 1);
      const int bmin = (nlo <= 0 && nhi >= 0) ? 0 : std::min(std::abs(nlo), std::abs(nhi));
      const int kb = std::max(std::max(mp, bmin), lmin);  // B rows l < lmin are zero
      if (kb >= Lb) continue;
      range[(size_t)mp * ntiles + t] = make_int2(kb / TC_CHUNK_K, nchunk - kb / TC_CHUNK_K);
    }
}

void tc_analysis_a_ranges(int Lb, int lmin, const ColSet& cs, std::vector<int2>& range, int& nmt) {
  nmt = (cs.Mc + TC_A_ROWS / 2 - 1) / (TC_A_ROWS / 2);
  const int nchunk = (Lb + TC_CHUNK_K - 1) / TC_CHUNK_K;
  range.assign((size_t)Lb * nmt, make_int2(0, 0));
  for (int mp = 0; mp < Lb; ++mp)
    for (int t = 0; t < nmt; ++t) {
      const int amin = tc_tile_amin(cs, t * (TC_A_ROWS / 2), TC_A_ROWS / 2);
      // the same lower limits as the B runs, so every chunk a tile visits is in its A run
      const int kb = std::max(std::max(mp, amin), lmin);
      if (kb >= Lb) continue;
      range[(size_t)mp * nmt + t] = make_int2(kb / TC_CHUNK_K, nchunk - kb / TC_CHUNK_K);
    }
}

void tc_synthesis_ranges(int Lb, int lmin, const ColSet& cs, std::vector<int2>& range, int& ntiles) {
  ntiles = (Lb + TC_TILE_ROWS - 1) / TC_TILE_ROWS;
  range.assign((size_t)Lb * ntiles, make_int2(0, 0));
  for (int mp = 0; mp < Lb; ++mp)
    for (int t = 0; t < ntiles; ++t) {
      const int lhi = std::min((t + 1) * TC_TILE_ROWS, Lb) - 1;
      if (mp > lhi || lhi < lmin) continue;  // every row l of the tile below the support: Z = 0
      const int d = -lhi - cs.n0, dmax = lhi - cs.n0;
      const int kb = d <= 0 ? 0 : (d + cs.nstep - 1) / cs.nstep;
      const int ke = dmax < 0 ? 0 : std::min(cs.Nc, dmax / cs.nstep + 1);
      if (ke <= kb) continue;
      const int c0 = kb / TC_CHUNK_K, c1 = (ke + TC_CHUNK_K - 1) / TC_CHUNK_K;
      range[(size_t)mp * ntiles + t] = make_int2(c0, c1 - c0);
    }
}

long long tc_check_ranges(int Lb, int lmin_b, int lmin_a, const ColSet& cs, long long* tiles) {
  static_assert(TC_A_ROWS == tc::BM && TC_TILE_ROWS == tc::BNC, "table tiles are engine tiles");
  std::vector<int2> rb, ra, rs;
  int nt = 0, nmt = 0, nts = 0;
  tc_analysis_ranges(Lb, lmin_b, cs, rb, nt);
  tc_analysis_a_ranges(Lb, lmin_a, cs, ra, nmt);
  tc_synthesis_ranges(Lb, lmin_b, cs, rs, nts);
  const int nchunk = (Lb + TC_CHUNK_K - 1) / TC_CHUNK_K, MR = TC_A_ROWS / 2;
  long long bad = 0, n = 0;
  for (int mp = 0; mp < Lb; ++mp)
    for (int by = 0; by < nmt; ++by) {
      const int amin = tc_tile_amin(cs, by * MR, MR);
      const int2 a = ra[(size_t)mp * nmt + by];
      for (int bx = 0; bx < nt; ++bx) {  // analysis: rows (m, Re|Im), columns n, K = l
        ++n;
        const int2 rg = rb[(size_t)mp * nt + bx];
        const int2 ch = tc_analysis_tile_chunks(rg, amin);
        const int nlo = cs.n0 + cs.nstep * (bx * TC_TILE_ROWS);
        const int nhi = cs.n0 + cs.nstep * (std::min((bx + 1) * TC_TILE_ROWS, cs.Nc) - 1);
        const int bmin = (nlo <= 0 && nhi >= 0) ? 0 : std::min(std::abs(nlo), std::abs(nhi));
        // lowest l of a nonzero product: l >= m', l >= |m|, l >= |n| and Psi_ln != 0
        const int need = std::max(std::max(mp, lmin_b), std::max(amin, bmin));
        bool ok = true;
        if (ch.y > ch.x) {
          ok = rg.x <= ch.x && ch.y <= rg.x + rg.y && ch.y <= nchunk && a.y > 0 && a.x <= ch.x &&
               ch.y <= a.x + a.y;
        }
        if (need < Lb) ok = ok && ch.y > ch.x && ch.x * TC_CHUNK_K <= need && ch.y == nchunk;
        if (!ok) ++bad;
      }
      for (int bx = 0; bx < nts; ++bx) {  // synthesis: rows (m, Re|Im), columns l, K = n
        ++n;
        const int2 rg = rs[(size_t)mp * nts + bx];
        const int llo = bx * TC_TILE_ROWS, lhi = std::min(llo + TC_TILE_ROWS, Lb) - 1;
        const bool work = !(amin > lhi) && rg.y > 0;  // the rule of SynthesisProb::tile
        // the reduction reads Z[m'][m][l] for l >= max(lmin, m', |m|)
        const bool read = std::max(std::max(lmin_b, llo), std::max(mp, amin)) <= lhi;
        bool ok = !read || work;
        if (read && work) {  // every n with |n| <= lhi inside the run
          const int d = -lhi - cs.n0, dmax = lhi - cs.n0;
          const int kb = d <= 0 ? 0 : (d + cs.nstep - 1) / cs.nstep;
          const int ke = dmax < 0 ? 0 : std::min(cs.Nc, dmax / cs.nstep + 1);
          ok = rg.x * TC_CHUNK_K <= kb && ke <= (rg.x + rg.y) * TC_CHUNK_K;
        }
        if (!ok) ++bad;
      }
    }
  if (tiles) *tiles = n;
  return bad;
}

bool tc_fill_analysis_table(const float* Q32, int Lmax, const float* psi, int Lb, ColSet cs, TcTab t, float* hi,
                            float* lo, cudaStream_t st) {
  dim3 g(t.ntiles, Lb);
  KTimer kt(K_MISC, st);
  tc::fill_analysis_table_kernel<<<g, 256, 0, st>>>(Q32, Lmax, psi, Lb, cs, t, hi, lo);
  kt.done();
  return launch_ok("fill_analysis_table_kernel");
}

bool tc_fill_synthesis_table(const float* Q32, int Lmax, const float* psi, int Lb, ColSet cs, TcTab t, float* hi,
                             float* lo, cudaStream_t st) {
  dim3 g(t.ntiles, Lb);
  KTimer kt(K_MISC, st);
  tc::fill_synthesis_table_kernel<<<g, 256, 0, st>>>(Q32, Lmax, psi, Lb, cs, t, hi, lo);
  kt.done();
  return launch_ok("fill_synthesis_table_kernel");
}

// The warp-specialised persistent engine is the default; CRV_TC_WS=0 selects the
// one-tile-per-CTA form (two CTAs per SM), kept for comparison.
static bool use_ws() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("CRV_TC_WS");
    v = (e && e[0] == '0') ? 0 : 1;
  }
  return v == 1;
}
static int sm_count() { return device_sms(); }

bool tc_analysis(const float* Q32, int Lmax, const cx<float>* flm, TcTab tb, int Lb, ColSet cs, cx<float>* X,
                 int* err, int* ctr, cudaStream_t st, TcATab ta) {
  tc::AnalysisProb pb{Q32, Lmax, flm, tb, Lb, cs, X};
  pb.split = tb.kmax * TC_CHUNK_K > TC_SPLIT_K;
  dim3 grid(tb.ntiles, (cs.Mc + tc::BM / 2 - 1) / (tc::BM / 2), Lb);
  if (ta.hi && use_ws()) {
    // A operand into its tables first (one pass over Delta and f), then both operands by copy
    {
      KTimer kt(K_TC_A, st);
      tc::fill_analysis_a_kernel<<<dim3(ta.nmt, Lb), TC_A_ROWS, 0, st>>>(Q32, Lmax, flm, Lb, cs, ta);
      kt.done();
      if (!launch_ok("fill_analysis_a_kernel")) return false;
    }
    tc::AnalysisProbA pa;
    static_cast<tc::AnalysisProb&>(pa) = pb;
    pa.ta = ta;
    return launch_tc_gemm_ws<tc::AnalysisProbA, tc::BNC>(pa, grid, sm_count(), ctr, err, st, K_TC_A);
  }
  if (use_ws()) return launch_tc_gemm_ws<tc::AnalysisProb, tc::BNC>(pb, grid, sm_count(), ctr, err, st, K_TC_A);
  return launch_tc_gemm<tc::AnalysisProb, tc::BNC>(pb, grid, err, st, K_TC_A);
}

bool tc_synthesis(const float* Q32, int Lmax, const cx<float>* Y, TcTab tb, int Lb, ColSet cs, cx<float>* Zscratch,
                  cx<double>* flm, int* err, int* ctr, cudaStream_t st) {
  tc::SynthesisProb pb{Y, tb, Lb, cs, Zscratch};
  dim3 grid(tb.ntiles, (cs.Mc + tc::BM / 2 - 1) / (tc::BM / 2), Lb);
  const bool ok = use_ws() ? launch_tc_gemm_ws<tc::SynthesisProb, tc::BNC>(pb, grid, sm_count(), ctr, err, st, K_TC_S)
                           : launch_tc_gemm<tc::SynthesisProb, tc::BNC>(pb, grid, err, st, K_TC_S);
  if (!ok) return false;
  dim3 g2((Lb + 255) / 256, cs.Mc);
  KTimer kt(K_TC_S, st);
  tc::synth_reduce_kernel<<<g2, 256, 0, st>>>(Q32, Lmax, Zscratch, Lb, tb.lmin, cs, flm);
  kt.done();
  return launch_ok("synth_reduce_kernel");
}

bool tc_bounded_wait_probe(int* err, long polls, cudaStream_t st) {
  tc::bounded_wait_probe_kernel<<<1, 32, 0, st>>>(err, polls);
  count_launch();
  return launch_ok("bounded_wait_probe_kernel");
}

}  // namespace crv
