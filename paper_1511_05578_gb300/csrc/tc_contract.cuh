// Interface of the tensor-core (tcgen05) split-FP32 Delta contractions of the mixed path
// (tc_contract.cu), used by crv.cu.
#pragma once
#include <vector>

#include "transforms.cuh"

namespace crv {

// Plan-constant B operand of one contraction and one scale: for every (m', tile) the run of
// 16-wide K chunks that the tile multiplies, each chunk a 256-row x 16 block in exactly the
// shared-memory layout of one stage of the tensor-core engine (rows in 8-row groups of 512 B,
// k-quads 128 B apart, 16 B per row and quad), already split into TF32 hi = rna(x) and
// lo = rna(x - hi), so that one bulk copy per half fills a stage.
//   analysis:  rows n (256 per tile), K = l,  value Delta^l_{m'n} Psi_ln
//   synthesis: rows l (256 per tile), K = ni, value Delta^l_{m'n} Psi_ln
// Chunk kc of (m', tile) sits at hi/lo + (base[m' * ntiles + tile] + kc) * TC_CHUNK_FLOATS;
// range[m' * ntiles + tile] = (first chunk, number of chunks); entries outside the support
// (l < max(m', |n|), l >= Lb, ni >= Nc) are zero.
struct TcTab {
  const float* hi = nullptr;
  const float* lo = nullptr;
  const long long* base = nullptr;
  const int2* range = nullptr;
  int ntiles = 0;
  int kmax = 0;  // the longest run of K chunks over (m', tile)
  int lmin = 0;  // first l of the scale's kernel support (Psi_ln = 0 below it)
};
constexpr int TC_TILE_ROWS = 256, TC_CHUNK_K = 16, TC_CHUNK_FLOATS = TC_TILE_ROWS * TC_CHUNK_K;
// The tensor core's FP32 accumulation behaves like truncation, so the error of a long K sum
// grows with the number of MMA steps into it (three per K-step of 8 with one accumulator).
// Analysis scales whose K runs exceed TC_SPLIT_K take the hi*hi products and the corrections
// in separate accumulators (one step per K-step at full size), at the cost of a single-
// buffered accumulator pair; the shorter runs stay double-buffered.
constexpr int TC_SPLIT_K = 512;

// Smallest |m| over the tile of `rows` values of m from column index mi0 (0 if it holds m = 0).
__host__ __device__ inline int tc_tile_amin(const ColSet& cs, int mi0, int rows) {
  const int mlo = cs.m0 + mi0, mend = mi0 + rows < cs.Mc ? mi0 + rows : cs.Mc, mhi = cs.m0 + mend - 1;
  const int alo = mlo < 0 ? -mlo : mlo, ahi = mhi < 0 ? -mhi : mhi;
  return (mlo <= 0 && mhi >= 0) ? 0 : (alo < ahi ? alo : ahi);
}
// K chunks [x, y) that an analysis tile multiplies: its B run rg from the m-tile's smallest |m|
// on (Delta^l_{m'm} = 0 for l < |m|); empty (x == y) when that lies past the run.
__host__ __device__ inline int2 tc_analysis_tile_chunks(int2 rg, int amin) {
  const int c0 = rg.x > amin / TC_CHUNK_K ? rg.x : amin / TC_CHUNK_K, c1 = rg.x + rg.y;
  return make_int2(c0, c1 > c0 ? c1 : c0);
}

// Per-map A operand of the analysis contraction for one scale (rebuilt for every map and
// scale): for every (m', m-tile of 64 values of m) the run of 16-wide K chunks from
// l = max(m', min |m| of the tile) on, each chunk a 128-row x 16 block (rows (m, Re|Im),
// value Delta^l_{m'm} f_lm) in an engine stage's layout, split into TF32 hi and lo. Chunk
// kc of (m', mt) sits at hi/lo + (base[m' * nmt + mt] + kc) * TC_ACHUNK_FLOATS.
constexpr int TC_A_ROWS = 128, TC_ACHUNK_FLOATS = TC_A_ROWS * TC_CHUNK_K;
struct TcATab {
  float* hi = nullptr;
  float* lo = nullptr;
  const long long* base = nullptr;
  const int2* range = nullptr;
  int nmt = 0;
};

// Chunk ranges per (m', tile), m' < Lb (host).
void tc_analysis_ranges(int Lb, int lmin, const ColSet& cs, std::vector<int2>& range, int& ntiles);
// Chunk ranges of the per-map A tables per (m', m-tile) (host).
void tc_analysis_a_ranges(int Lb, int lmin, const ColSet& cs, std::vector<int2>& range, int& nmt);
void tc_synthesis_ranges(int Lb, int lmin, const ColSet& cs, std::vector<int2>& range, int& ntiles);
// Host check of one scale's runs as the plan builds them (B runs from lmin_b, A runs from
// lmin_a; a plan uses one lmin for both) against the engines' tile rules: every analysis tile
// with work stays inside its B and A runs and covers every l >= lmin_b its products need,
// and every synthesis tile whose Z the m' reduction reads has work covering its n. Returns the
// number of tiles that break a rule; *tiles gets the number checked.
long long tc_check_ranges(int Lb, int lmin_b, int lmin_a, const ColSet& cs, long long* tiles);
// Fill a table (device); t.base / t.range already on the device.
bool tc_fill_analysis_table(const float* Q32, int Lmax, const float* psi, int Lb, ColSet cs, TcTab t, float* hi,
                            float* lo, cudaStream_t st);
bool tc_fill_synthesis_table(const float* Q32, int Lmax, const float* psi, int Lb, ColSet cs, TcTab t, float* hi,
                             float* lo, cudaStream_t st);

// err: device error flag (bounded waits); ctr: a device int for the tile counter of the
// persistent engine (the plan's, one stream at a time).
bool tc_analysis(const float* Q32, int Lmax, const cx<float>* flm, TcTab tb, int Lb, ColSet cs, cx<float>* X,
                 int* err, int* ctr, cudaStream_t st, TcATab ta = TcATab());
bool tc_synthesis(const float* Q32, int Lmax, const cx<float>* Y, TcTab tb, int Lb, ColSet cs, cx<float>* Zscratch,
                  cx<double>* flm, int* err, int* ctr, cudaStream_t st);
// One thread waits on an mbarrier nothing arrives at, `polls` polls at most, and sets *err.
bool tc_bounded_wait_probe(int* err, long polls, cudaStream_t st);

}  // namespace crv
