// Launches of the double-float FFT kernels for one length (df_fft.cuh), instantiated by
// df_fft.cu (P = 4096) and df_fft2048.cu (P = 2048), one translation unit per length so that
// they build in parallel. Launch configuration as for the FP64 kernels: blocks of 256 threads,
// 256 / (P / 16) transforms (or column pairs) per block, one block per SM, grid-strided work.
#pragma once
#include <algorithm>

#include "df_fft.cuh"

namespace crv {
namespace dfimpl {

constexpr int NT = 256;

template <int P, bool COLS, class Ld, class St>
bool launch_dft(int kind, const DftTab<df>& tb, int sign, int nseq, Ld ld, St st, cudaStream_t s) {
  if (nseq <= 0) return true;
  if (tb.P != P) return false;
  auto kern = dft_kernel<df, NT, COLS, P, Ld, St>;
  const size_t smem = fft_smem_bytes<df>(NT);
  if (!func_attr_once((const void*)kern, (int)smem)) return false;
  carveout_for((const void*)kern, smem, 1);
  constexpr int G = NT / (P / 16);
  const int grid = std::max(1, std::min((nseq + G - 1) / G, device_sms()));
  KTimer kt(kind, s);
  kern<<<grid, NT, smem, s>>>(tb, sign, nseq, ld, st);
  kt.done();
  return launch_ok(kind_name(kind));
}

template <int P>
bool beta_synth(const DftTab<df>& tb, int Lb, int ncols, const cx<df>* X, cx<df>* Y, ColSet cs, cudaStream_t s) {
  if (ncols <= 0) return true;
  if (tb.P != P) return false;
  const size_t smem = fft_smem_bytes_tabs<df>(NT, P, 1);
  if (!func_attr_once((const void*)beta_synth_kernel<df, NT, P>, (int)smem)) return false;
  const int npair = num_col_pairs(cs);
  if (npair <= 0) return true;
  constexpr int G = NT / (P / 16);
  const int grid = std::max(1, std::min((npair + G - 1) / G, device_sms()));
  KTimer kt(K_BETA_SYNTH, s);
  beta_synth_kernel<df, NT, P><<<grid, NT, smem, s>>>(tb, ncols, Lb, X, Y, cs, PairMap());
  kt.done();
  return launch_ok("beta_synth_kernel (double-float)");
}

template <int P>
bool beta_quad(const DftTab<df>& tb, const CorrTab<df>& ct, int Lb, int ncols, const cx<df>* Xb, cx<df>* Y,
               ColSet cs, df scale, int pa, int pb, int pc, cudaStream_t s) {
  if (ncols <= 0) return true;
  if (tb.P != P || ct.Q != P) return false;
  const size_t smem = fft_smem_bytes_tabs<df>(NT, P, 2);
  if (!func_attr_once((const void*)beta_quad_kernel<df, NT, P>, (int)smem)) return false;
  const int npair = num_col_pairs(cs);
  if (npair <= 0) return true;
  constexpr int G = NT / (P / 16);
  const int grid = std::max(1, std::min((npair + G - 1) / G, device_sms()));
  KTimer kt(K_BETA_QUAD, s);
  beta_quad_kernel<df, NT, P><<<grid, NT, smem, s>>>(tb, ct, ncols, Lb, Xb, Y, cs, scale, pa, pb, pc, PairMap());
  kt.done();
  return launch_ok("beta_quad_kernel (double-float)");
}

}  // namespace dfimpl
}  // namespace crv

// The exported launches for one length P (df_fft.cuh declares them).
#define CRV_DF_DEFINE(P)                                                                                           \
  namespace crv {                                                                                                  \
  bool df_ring_m_##P(const DftTab<df>& tb, int n, LdRingMHalf<df, false> ld, StRingMHalf<df> st, cudaStream_t s) { \
    return dfimpl::launch_dft<P, true>(K_RING_INV_M, tb, +1, n, ld, st, s);                                        \
  }                                                                                                                \
  bool df_ring_n_##P(const DftTab<df>& tb, int n, LdRingNHerm<df, false> ld, StWRowPair<df, double> st,             \
                     cudaStream_t s) {                                                                             \
    return dfimpl::launch_dft<P, false>(K_RING_INV_N, tb, +1, n, ld, st, s);                                       \
  }                                                                                                                \
  bool df_ring_g_##P(const DftTab<df>& tb, int n, LdWRowPair<df, double> ld, StRingNPairHalf<df> st,              \
                     cudaStream_t s) {                                                                             \
    return dfimpl::launch_dft<P, false>(K_RING_FWD_G, tb, -1, n, ld, st, s);                                       \
  }                                                                                                                \
  bool df_ring_a_##P(const DftTab<df>& tb, int n, LdRingAHalf<df> ld, StRingAHalf<df> st, cudaStream_t s) {        \
    return dfimpl::launch_dft<P, true>(K_RING_FWD_A, tb, -1, n, ld, st, s);                                        \
  }                                                                                                                \
  bool df_beta_synth_##P(const DftTab<df>& tb, int Lb, int ncols, const cx<df>* X, cx<df>* Y, ColSet cs,           \
                         cudaStream_t s) {                                                                         \
    return dfimpl::beta_synth<P>(tb, Lb, ncols, X, Y, cs, s);                                                      \
  }                                                                                                                \
  bool df_beta_quad_##P(const DftTab<df>& tb, const CorrTab<df>& ct, int Lb, int ncols, const cx<df>* Xb,          \
                        cx<df>* Y, ColSet cs, df scale, int pa, int pb, int pc, cudaStream_t s) {                  \
    return dfimpl::beta_quad<P>(tb, ct, Lb, ncols, Xb, Y, cs, scale, pa, pb, pc, s);                               \
  }                                                                                                                \
  }
