// Rotation of Wigner coefficients (Sec. III-A-1, Eqs. curvelet_Wigner, curvelet_Wigner_inverse,
// rotateWigner). With rho* = (0, vartheta^j, 0), W(rho) = W~(rho rho*) and
// D^l(rho rho*) = D^l(rho) D^l(rho*) give (W)^l_mk = sum_n (W~)^l_mn d^l_kn(vartheta); the
// unrotated coefficients vanish unless |n| = l (Eq. curvelet_Wigner_property), so each rotated
// coefficient takes two terms and a scale costs O(L_j^3). d^l_{k,-l} = (-1)^{l+k} d^l_{-k,l}
// comes from the same edge column d^l_{k,l}(vartheta). FP64 throughout.
#include "rotate.cuh"

namespace crv {

__global__ void __launch_bounds__(128) rotate_wigner_kernel(const double* __restrict__ edge, int Lj,
                                                            const cx<double>* __restrict__ wt,
                                                            cx<double>* __restrict__ w) {
  const int N = 2 * Lj - 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x, mi = blockIdx.y, l = blockIdx.z;
  if (k >= N) return;
  const int m = mi - (Lj - 1), kk = k - (Lj - 1);
  cx<double> out = mk(0.0, 0.0);
  if (abs(m) <= l && abs(kk) <= l) {
    out = wt[(size_t)l * N + mi] * edge[(size_t)l * N + k];
    if (l > 0) {
      const double dm = edge[(size_t)l * N + (Lj - 1 - kk)] * parity_sign(l + kk);
      out = out + wt[(size_t)(Lj + l) * N + mi] * dm;
    }
  }
  w[((size_t)l * N + mi) * N + k] = out;
}

// One block per (m, l): the two sums over k, reduced in a fixed order (deterministic).
__global__ void __launch_bounds__(128) rotate_wigner_adjoint_kernel(const double* __restrict__ edge, int Lj,
                                                                    const cx<double>* __restrict__ w,
                                                                    cx<double>* __restrict__ wt) {
  const int N = 2 * Lj - 1;
  const int mi = blockIdx.x, l = blockIdx.y, m = mi - (Lj - 1);
  __shared__ cx<double> red[2][4];
  cx<double> sp = mk(0.0, 0.0), sm = mk(0.0, 0.0);
  if (abs(m) <= l) {
    const cx<double>* row = w + ((size_t)l * N + mi) * N;
    for (int kk = -l + (int)threadIdx.x; kk <= l; kk += blockDim.x) {
      const int k = kk + Lj - 1;
      const cx<double> v = row[k];
      sp = sp + v * edge[(size_t)l * N + k];
      sm = sm + v * (edge[(size_t)l * N + (Lj - 1 - kk)] * parity_sign(l + kk));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sp.re += __shfl_xor_sync(0xffffffffu, sp.re, o);
    sp.im += __shfl_xor_sync(0xffffffffu, sp.im, o);
    sm.re += __shfl_xor_sync(0xffffffffu, sm.re, o);
    sm.im += __shfl_xor_sync(0xffffffffu, sm.im, o);
  }
  const int wp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][wp] = sp; red[1][wp] = sm; }
  __syncthreads();
  if (threadIdx.x == 0) {
    cx<double> a = red[0][0], b = red[1][0];
    for (int i = 1; i < 4; ++i) { a = a + red[0][i]; b = b + red[1][i]; }
    const bool in = abs(m) <= l;
    wt[(size_t)l * N + mi] = in ? a : mk(0.0, 0.0);
    wt[(size_t)(Lj + l) * N + mi] = (in && l > 0) ? b : mk(0.0, 0.0);
  }
}

bool rotate_wigner_launch(const double* edge, int Lj, const cx<double>* wt, cx<double>* w, cudaStream_t st) {
  const int N = 2 * Lj - 1;
  KTimer kt(K_ROTATE, st);
  rotate_wigner_kernel<<<dim3((N + 127) / 128, N, Lj), 128, 0, st>>>(edge, Lj, wt, w);
  kt.done();
  return launch_ok("rotate_wigner_kernel");
}

bool rotate_wigner_adjoint_launch(const double* edge, int Lj, const cx<double>* w, cx<double>* wt, cudaStream_t st) {
  const int N = 2 * Lj - 1;
  KTimer kt(K_ROTATE, st);
  rotate_wigner_adjoint_kernel<<<dim3(N, Lj), 128, 0, st>>>(edge, Lj, w, wt);
  kt.done();
  return launch_ok("rotate_wigner_adjoint_kernel");
}

}  // namespace crv
