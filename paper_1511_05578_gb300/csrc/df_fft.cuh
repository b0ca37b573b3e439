// Launches of the double-float FFT kernels of the FP64 plans (df_fft.cu): the P = 4096 Wigner
// transforms of real signals with FP64 coefficients, the same steps as the FP64 kernels in
// double-float arithmetic (df in common.cuh). All on stream s; false on a launch error.
#pragma once
#include "transforms.cuh"

namespace crv {

// Ring steps: m step (analysis, sign +1, columns), n step with real output (analysis, +1,
// rows), g step on real row pairs (synthesis, -1, rows), a step (synthesis, -1, columns).
bool df_ring_m(const DftTab<df>& tb, int nseq, LdRingMHalf<df, false> ld, StRingMHalf<df> st, cudaStream_t s);
bool df_ring_n(const DftTab<df>& tb, int nseq, LdRingNHerm<df, false> ld, StWRowPair<df, double> st,
               cudaStream_t s);
bool df_ring_g(const DftTab<df>& tb, int nseq, LdWRowPair<df, double> ld, StRingNPairHalf<df> st, cudaStream_t s);
bool df_ring_a(const DftTab<df>& tb, int nseq, LdRingAHalf<df> ld, StRingAHalf<df> st, cudaStream_t s);
// Beta transforms of all column pairs (no pair list: rotated coefficients).
bool df_beta_synth(const DftTab<df>& tb, int Lb, int ncols, const cx<df>* X, cx<df>* Y, ColSet cs, cudaStream_t s);
bool df_beta_quad(const DftTab<df>& tb, const CorrTab<df>& ct, int Lb, int ncols, const cx<df>* Xb, cx<df>* Y,
                  ColSet cs, df scale, int pa, int pb, int pc, cudaStream_t s);

}  // namespace crv
