// fv_learned.cuh — face states of the learned-stencil step (shallow water),
// shared by the two-pass learned step (CNN, then stage kernel) and the fused
// row-pipelined kernel, so both evaluate the same arithmetic per face.
//
// Section 2.5.3, fourth approach: the owner cell's normalised coefficients
// give Q^L = wL0 Q_{i-1} + wL1 Q_i + wL2 Q_{i+1} and
// Q^R = wR0 Q_i + wR1 Q_{i+1} + wR2 Q_{i+2}; where a learned depth falls below
// h_min the face takes the MUSCL-minmod states (Eq. 2.18) instead.
#pragma once

#include "fv_common.cuh"

namespace fvk {

// Learned (or, below h_min, minmod) face states of one face from its 4-cell
// stencil m = Q_{i-1}, a = Q_i, b = Q_{i+1}, p = Q_{i+2} and the owner's 18
// coefficients of this direction, wd[(var * 2 + side) * 3 + tap].
__device__ __forceinline__ void learned_face(const float (&m)[3], const float (&a)[3],
                                             const float (&b)[3], const float (&p)[3],
                                             const float (&wd)[18], float hmin, float (&L)[3],
                                             float (&R)[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* wl = wd + (c * 2 + 0) * 3;
    const float* wr = wd + (c * 2 + 1) * 3;
    L[c] = vfma(wl[2], b[c], vfma(wl[1], a[c], vmul(wl[0], m[c])));
    R[c] = vfma(wr[2], p[c], vfma(wr[1], b[c], vmul(wr[0], a[c])));
  }
  if (!(L[0] >= hmin) || !(R[0] >= hmin)) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      L[c] = face_left(a[c], minmod(vsub(a[c], m[c]), vsub(b[c], a[c])));
      R[c] = face_right(b[c], minmod(vsub(b[c], a[c]), vsub(p[c], b[c])));
    }
  }
}

}  // namespace fvk
