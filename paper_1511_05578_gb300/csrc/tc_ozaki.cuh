// Interface of the FP64-accurate tensor-core Delta contractions (tc_ozaki.cu), used by crv.cu
// for plans with CRV_F_FP64_TC.
//
// The contractions are those of the plain FP64 path (Eq. inverse_Fmnmp in general-n form with
// Eq. wav_harmonic_coeff folded in; Eq. flml in general-n form with the n-sum of Eq.
// wav_synthesis_harmonic), computed as products of integer slices on the TF32 tensor cores
// with the integer sums exact in FP32 accumulators (the error-free splitting of Ozaki et al.):
// every row x of an operand (over K) gets a power-of-two scale 2^E > max |x| and is written
// with b-bit digits as
//   x = 2^(E - b + 1) sum_{k < OZ_S} d_k 2^(-bk),   d_k integers in [-2^(b-1), 2^(b-1)],
// and slice k holds d_k 2^(-bk) (exact in TF32). A product of slices s, t carries 2^(-b(s+t));
// the products of one level s + t <= OZ_EXACT_LEVELS - 1 go to an FP32 accumulator of their
// own, where a sum over K of at most four of them stays an integer multiple of 2^(-b(s+t))
// of magnitude <= 4 K 2^(2b-2) <= 2^24 of those: exact for b = 7 and K <= 1024 (every l
// range, and every n range of real signals) and for b = 6 and K <= 2048 (the n ranges of
// complex signals above L = 512), the plan taking the larger b that holds. The levels above,
// of weight 2^(-4b) and less, share one more accumulator; levels above OZ_S - 1 are dropped.
// The dropped products (levels >= OZ_S, random digits) leave an error of at most about
// 2^(-b OZ_S + 8) sqrt(K) max|A| max|B| per element: 2^-36 sqrt(K) for b = 7, 2^-29 sqrt(K)
// for b = 6, relative to the largest possible term. The epilogue adds the accumulators in double-float and scales by
// 2^(Ea + Eb - 2b + 2) into FP64.
#pragma once
#include <vector>

#include "transforms.cuh"

namespace crv {

constexpr int OZ_S = 7;              // slices per operand row
constexpr int OZ_EXACT_LEVELS = 4;   // levels 0..3 each in an exact accumulator
constexpr int OZ_ACCS = OZ_EXACT_LEVELS + 1;
constexpr int OZ_K = 16;             // K per chunk (one engine stage)
constexpr int OZ_AROWS = 128;        // A tile rows: 64 values of m, Re and Im
constexpr int OZ_BROWS = 96;         // B tile rows = accumulator columns
constexpr int OZ_ASLICE = OZ_AROWS * OZ_K, OZ_BSLICE = OZ_BROWS * OZ_K;  // floats per slice of a chunk
constexpr int OZ_ACHUNK = OZ_S * OZ_ASLICE, OZ_BCHUNK = OZ_S * OZ_BSLICE;

// A sliced operand table for one scale: for every (m', tile) the run of K chunks that the
// tile multiplies, each chunk OZ_S slices of a (rows x 16) block in the layout of an engine
// stage (8-row groups of 512 B, k-quads 128 B apart, 16 B per row and quad). Chunk kc of
// (m', tile) sits at v + (base[(m' - mp0) * ntiles + tile] - c0 + kc) * chunk floats;
// range[(m' - mp0) * ntiles + tile] = (first chunk, number of chunks); the row scales are
// e[(m' - mp0) * rows + row]. Tables of the per-map A operands hold the m' in [mp0, mp1)
// (one pass of the engine), c0 being the chunk offset of mp0 in the scale's layout.
struct OzTab {
  float* v = nullptr;
  int* e = nullptr;
  const long long* base = nullptr;
  const int2* range = nullptr;
  int ntiles = 0, rows = 0, mp0 = 0, mp1 = 0;
  long long c0 = 0;
  int bits = 7;  // digit width b (the same for both operands of a contraction)
};

// Chunk ranges (host), over all m' < Lb: B tables (analysis: rows n, K = l; synthesis: rows
// l, K = ni) per (m', tile of OZ_BROWS rows); A tables (analysis: rows (m, Re|Im), K = l;
// synthesis: K = ni) per (m', tile of 64 m).
void oz_ranges_b_analysis(int Lb, const ColSet& cs, std::vector<int2>& range, int& ntiles);
void oz_ranges_b_synthesis(int Lb, const ColSet& cs, std::vector<int2>& range, int& ntiles);
void oz_ranges_a_analysis(int Lb, const ColSet& cs, std::vector<int2>& range, int& ntiles);
void oz_ranges_a_synthesis(int Lb, const ColSet& cs, std::vector<int2>& range, int& ntiles);

// Plan-time B tables (Delta^l_{m'n} Psi_ln, FP64 inputs).
bool oz_fill_b_analysis(const double* Q, int Lmax, const double* psi, int Lb, ColSet cs, OzTab t, cudaStream_t st);
bool oz_fill_b_synthesis(const double* Q, int Lmax, const double* psi, int Lb, ColSet cs, OzTab t, cudaStream_t st);

// Analysis of the m' in [ta.mp0, ta.mp1): fills the A table from f_lm, then X planes of those m'.
bool oz_analysis(const double* Q, int Lmax, const cx<double>* flm, OzTab ta, OzTab tb, int Lb, ColSet cs,
                 cx<double>* X, int* err, int* ctr, cudaStream_t st);
// Synthesis products of the m' in [ta.mp0, ta.mp1): fills the A table from Y', then
// Z[m'][mi][l] = sum_n Y'_{m n m'} Delta^l_{m'n} Psi_ln for those m'.
bool oz_synthesis_products(const cx<double>* Y, OzTab ta, OzTab tb, int Lb, ColSet cs, cx<double>* Z, int* err,
                           int* ctr, cudaStream_t st);
// f_lm += sum_{m' <= l} Delta^l_{m'm} Z[m'][mi][l] in FP64 (Eq. flml's sum over m').
bool oz_synthesis_reduce(const double* Q, int Lmax, const cx<double>* Z, int Lb, ColSet cs, cx<double>* flm,
                         cudaStream_t st);

}  // namespace crv
