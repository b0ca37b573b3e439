// Rotation of Wigner coefficients between the unrotated and the rotated curvelet
// coefficients of one scale (Sec. III-A-1; used by crv.cu).
#pragma once
#include "common.cuh"

namespace crv {

// (W)^l_mk = (W~)^l_{m,l} d^l_{k,l}(vartheta) + (W~)^l_{m,-l} d^l_{k,-l}(vartheta), dense in (m, k).
//   edge [Lj][2Lj-1]: d^l_{k,l}(vartheta) at k + Lj - 1 (zero for |k| > l)
//   wt   [2][Lj][2Lj-1]: (W~)^l_{m,+l}, (W~)^l_{m,-l} at m + Lj - 1
//   w    [Lj][2Lj-1][2Lj-1]
bool rotate_wigner_launch(const double* edge, int Lj, const cx<double>* wt, cx<double>* w, cudaStream_t st);
// (W~)^l_{m,+-l} = sum_k (W)^l_mk d^l_{k,+-l}(vartheta), the adjoint (and inverse on rotated
// coefficients); wt[1][0][.] = 0.
bool rotate_wigner_adjoint_launch(const double* edge, int Lj, const cx<double>* w, cx<double>* wt, cudaStream_t st);

}  // namespace crv
