// The double-float FFT kernels of the FP64 plans (see df in common.cuh), compiled in a
// translation unit of their own so that they build in parallel with crv.cu: the largest Wigner
// FFT length (P = 4096, band limit 1024) of real signals with FP64 coefficients -- the four
// ring steps and the two beta transforms. Every other length and signal keeps the FP64 kernels.
// Launch configuration as for the FP64 kernels: blocks of 256 threads, one transform (or column
// pair) each, one block per SM, a grid of at most one block per SM striding through the work.
#include <algorithm>

#include "df_fft.cuh"

namespace crv {

namespace {
constexpr int NT = 256, P = 4096;

template <bool COLS, class Ld, class St>
bool launch_dft(int kind, const DftTab<df>& tb, int sign, int nseq, Ld ld, St st, cudaStream_t s) {
  if (nseq <= 0) return true;
  if (tb.P != P) return false;
  auto kern = dft_kernel<df, NT, COLS, P, Ld, St>;
  const size_t smem = fft_smem_bytes<df>(NT);
  if (!func_attr_once((const void*)kern, (int)smem)) return false;
  carveout_for((const void*)kern, smem, 1);
  const int grid = std::max(1, std::min(nseq, device_sms()));  // one transform per block
  KTimer kt(kind, s);
  kern<<<grid, NT, smem, s>>>(tb, sign, nseq, ld, st);
  kt.done();
  return launch_ok(kind_name(kind));
}
}  // namespace

bool df_ring_m(const DftTab<df>& tb, int nseq, LdRingMHalf<df, false> ld, StRingMHalf<df> st, cudaStream_t s) {
  return launch_dft<true>(K_RING_INV_M, tb, +1, nseq, ld, st, s);
}
bool df_ring_n(const DftTab<df>& tb, int nseq, LdRingNHerm<df, false> ld, StWRowPair<df, double> st,
               cudaStream_t s) {
  return launch_dft<false>(K_RING_INV_N, tb, +1, nseq, ld, st, s);
}
bool df_ring_g(const DftTab<df>& tb, int nseq, LdWRowPair<df, double> ld, StRingNPairHalf<df> st, cudaStream_t s) {
  return launch_dft<false>(K_RING_FWD_G, tb, -1, nseq, ld, st, s);
}
bool df_ring_a(const DftTab<df>& tb, int nseq, LdRingAHalf<df> ld, StRingAHalf<df> st, cudaStream_t s) {
  return launch_dft<true>(K_RING_FWD_A, tb, -1, nseq, ld, st, s);
}

bool df_beta_synth(const DftTab<df>& tb, int Lb, int ncols, const cx<df>* X, cx<df>* Y, ColSet cs, cudaStream_t s) {
  if (ncols <= 0) return true;
  if (tb.P != P) return false;
  const size_t smem = fft_smem_bytes_tabs<df>(NT, P, 1);
  if (!func_attr_once((const void*)beta_synth_kernel<df, NT, P>, (int)smem)) return false;
  const int npair = num_col_pairs(cs);
  if (npair <= 0) return true;
  const int grid = std::max(1, std::min(npair, device_sms()));
  KTimer kt(K_BETA_SYNTH, s);
  beta_synth_kernel<df, NT, P><<<grid, NT, smem, s>>>(tb, ncols, Lb, X, Y, cs, PairMap());
  kt.done();
  return launch_ok("beta_synth_kernel (double-float)");
}

bool df_beta_quad(const DftTab<df>& tb, const CorrTab<df>& ct, int Lb, int ncols, const cx<df>* Xb, cx<df>* Y,
                  ColSet cs, df scale, int pa, int pb, int pc, cudaStream_t s) {
  if (ncols <= 0) return true;
  if (tb.P != P || ct.Q != P) return false;
  const size_t smem = fft_smem_bytes_tabs<df>(NT, P, 2);
  if (!func_attr_once((const void*)beta_quad_kernel<df, NT, P>, (int)smem)) return false;
  const int npair = num_col_pairs(cs);
  if (npair <= 0) return true;
  const int grid = std::max(1, std::min(npair, device_sms()));
  KTimer kt(K_BETA_QUAD, s);
  beta_quad_kernel<df, NT, P><<<grid, NT, smem, s>>>(tb, ct, ncols, Lb, Xb, Y, cs, scale, pa, pb, pc, PairMap());
  kt.done();
  return launch_ok("beta_quad_kernel (double-float)");
}

}  // namespace crv
