// Launches of the double-float FFT kernels of the FP64 plans: the Wigner transforms of real
// signals with FP64 coefficients at the two largest lengths (P = 4096 and 2048, band limits up
// to 1024 and 512), the same steps as the FP64 kernels in double-float arithmetic (df in
// common.cuh), each length compiled in a translation unit of its own (df_fft.cu,
// df_fft2048.cu). All on stream s; false on a launch error or another length.
#pragma once
#include "transforms.cuh"

namespace crv {

#define CRV_DF_DECLARE(P)                                                                                          \
  bool df_ring_m_##P(const DftTab<df>& tb, int n, LdRingMHalf<df, false> ld, StRingMHalf<df> st, cudaStream_t s); \
  bool df_ring_n_##P(const DftTab<df>& tb, int n, LdRingNHerm<df, false> ld, StWRowPair<df, double> st,            \
                     cudaStream_t s);                                                                              \
  bool df_ring_g_##P(const DftTab<df>& tb, int n, LdWRowPair<df, double> ld, StRingNPairHalf<df> st,              \
                     cudaStream_t s);                                                                              \
  bool df_ring_a_##P(const DftTab<df>& tb, int n, LdRingAHalf<df> ld, StRingAHalf<df> st, cudaStream_t s);        \
  bool df_beta_synth_##P(const DftTab<df>& tb, int Lb, int ncols, const cx<df>* X, cx<df>* Y, ColSet cs,          \
                         cudaStream_t s);                                                                          \
  bool df_beta_quad_##P(const DftTab<df>& tb, const CorrTab<df>& ct, int Lb, int ncols, const cx<df>* Xb,         \
                        cx<df>* Y, ColSet cs, df scale, int pa, int pb, int pc, cudaStream_t s);
CRV_DF_DECLARE(4096)
CRV_DF_DECLARE(2048)
#undef CRV_DF_DECLARE

// Ring steps: m step (analysis, sign +1, columns), n step with real output (analysis, +1, rows),
// g step on real row pairs (synthesis, -1, rows), a step (synthesis, -1, columns); beta
// transforms of all column pairs. Each picks the kernels of the table's length.
inline bool df_ring_m(const DftTab<df>& tb, int n, LdRingMHalf<df, false> ld, StRingMHalf<df> st, cudaStream_t s) {
  return tb.P == 4096 ? df_ring_m_4096(tb, n, ld, st, s) : tb.P == 2048 && df_ring_m_2048(tb, n, ld, st, s);
}
inline bool df_ring_n(const DftTab<df>& tb, int n, LdRingNHerm<df, false> ld, StWRowPair<df, double> st,
                      cudaStream_t s) {
  return tb.P == 4096 ? df_ring_n_4096(tb, n, ld, st, s) : tb.P == 2048 && df_ring_n_2048(tb, n, ld, st, s);
}
inline bool df_ring_g(const DftTab<df>& tb, int n, LdWRowPair<df, double> ld, StRingNPairHalf<df> st,
                      cudaStream_t s) {
  return tb.P == 4096 ? df_ring_g_4096(tb, n, ld, st, s) : tb.P == 2048 && df_ring_g_2048(tb, n, ld, st, s);
}
inline bool df_ring_a(const DftTab<df>& tb, int n, LdRingAHalf<df> ld, StRingAHalf<df> st, cudaStream_t s) {
  return tb.P == 4096 ? df_ring_a_4096(tb, n, ld, st, s) : tb.P == 2048 && df_ring_a_2048(tb, n, ld, st, s);
}
inline bool df_beta_synth(const DftTab<df>& tb, int Lb, int ncols, const cx<df>* X, cx<df>* Y, ColSet cs,
                          cudaStream_t s) {
  return tb.P == 4096 ? df_beta_synth_4096(tb, Lb, ncols, X, Y, cs, s)
                      : tb.P == 2048 && df_beta_synth_2048(tb, Lb, ncols, X, Y, cs, s);
}
inline bool df_beta_quad(const DftTab<df>& tb, const CorrTab<df>& ct, int Lb, int ncols, const cx<df>* Xb, cx<df>* Y,
                         ColSet cs, df scale, int pa, int pb, int pc, cudaStream_t s) {
  return tb.P == 4096 ? df_beta_quad_4096(tb, ct, Lb, ncols, Xb, Y, cs, scale, pa, pb, pc, s)
                      : tb.P == 2048 && df_beta_quad_2048(tb, ct, Lb, ncols, Xb, Y, cs, scale, pa, pb, pc, s);
}

}  // namespace crv
