// fv_schemes.cuh — the numerical fluxes other than HLL (Section 2.3.3) for
// two states in the face frame (component 1 = normal momentum, 2 =
// tangential), shallow water (h, hu, hv) and Euler (rho, rho u, rho v, E):
//   Lax-Friedrichs (Eq. 2.11), Rusanov (Eq. 2.12), Roe (Eqs. 2.13-2.14),
//   HLLE (Eq. 2.16) and HLLC (Eq. 2.17),
// with the readings where the paper is silent: Lax-Friedrichs viscosity
// d / (4 dt) per direction of the unsplit 2D update; Rusanov speed the larger
// spectral radius |u| + c; Roe-averaged states with no entropy fix; HLLE
// speeds clamped by the Roe state's and by 0; HLLC with the outer speeds of
// HLL (Davis) and the middle speed from the jump conditions (Toro).
#pragma once

#include "fv_common.cuh"

namespace fvk {

enum Flux { FLUX_HLL = 0, FLUX_RUSANOV = 1, FLUX_LF = 2, FLUX_ROE = 3, FLUX_HLLE = 4, FLUX_HLLC = 5 };

// Physical x flux, normal velocity and sound speed of one face-frame state.
template <int C, int EQ>
__device__ __forceinline__ void frame_state(const float (&q)[C], float phys, float (&F)[C], float& u,
                                            float& c, float& p) {
  const float r = vrcp(q[0]);
  u = vmul(q[1], r);
  if constexpr (EQ == SWE) {
    const float gh = vmul(phys, q[0]);
    c = vsqrt(gh);
    p = vmul(vmul(0.5f, gh), q[0]);
    F[0] = q[1];
    F[1] = vfma(q[1], u, p);
    F[2] = vmul(q[2], u);
  } else {
    const float v = vmul(q[2], r);
    p = vmul(phys - 1.f, vfma(-0.5f, vfma(q[1], u, vmul(q[2], v)), q[3]));
    c = vsqrt(vmul(vmul(phys, p), r));
    F[0] = q[1];
    F[1] = vfma(q[1], u, p);
    F[2] = vmul(q[2], u);
    F[3] = vmul(u, vadd(q[3], p));
  }
}

// 1/2 (F_L + F_R) - nu (Q_R - Q_L)
template <int C>
__device__ __forceinline__ void central(const float (&FL)[C], const float (&FR)[C], const float (&L)[C],
                                        const float (&R)[C], float nu, float (&F)[C]) {
#pragma unroll
  for (int k = 0; k < C; ++k) F[k] = vsub(vmul(0.5f, vadd(FL[k], FR[k])), vmul(nu, vsub(R[k], L[k])));
}

// Roe-averaged u, v, c (and H for Euler) of two face-frame states.
template <int C, int EQ>
__device__ __forceinline__ void roe_state(const float (&L)[C], const float (&R)[C], float phys, float& u,
                                          float& v, float& c, float& H, float pL, float pR) {
  const float sL = vsqrt(L[0]), sR = vsqrt(R[0]);
  const float w = vrcp(vadd(sL, sR));
  u = vmul(vadd(vmul(L[1], vrcp(sL)), vmul(R[1], vrcp(sR))), w);
  v = vmul(vadd(vmul(L[2], vrcp(sL)), vmul(R[2], vrcp(sR))), w);
  if constexpr (EQ == SWE) {
    c = vsqrt(vmul(phys, vmul(0.5f, vadd(L[0], R[0]))));
    H = 0.f;
  } else {
    const float HL = vmul(vadd(L[3], pL), vrcp(L[0]));
    const float HR = vmul(vadd(R[3], pR), vrcp(R[0]));
    H = vmul(vadd(vmul(sL, HL), vmul(sR, HR)), w);
    c = vsqrt(vmul(phys - 1.f, vsub(H, vmul(0.5f, vfma(u, u, vmul(v, v))))));
  }
}

template <int C, int EQ>
__device__ __forceinline__ void roe_flux(const float (&L)[C], const float (&R)[C], const float (&FL)[C],
                                         const float (&FR)[C], float pL, float pR, float phys,
                                         float (&F)[C]) {
  float u, v, c, H;
  roe_state<C, EQ>(L, R, phys, u, v, c, H, pL, pR);
  float d[C];
#pragma unroll
  for (int k = 0; k < C; ++k) d[k] = vsub(R[k], L[k]);
  const float l1 = fabsf(vsub(u, c)), l2 = fabsf(u), l3 = fabsf(vadd(u, c));
  const float r2c = vrcp(vadd(c, c));
  float D[C];
  if constexpr (EQ == SWE) {
    const float a1 = vmul(vsub(vmul(vadd(u, c), d[0]), d[1]), r2c);
    const float a3 = vmul(vsub(d[1], vmul(vsub(u, c), d[0])), r2c);
    const float a2 = vsub(d[2], vmul(v, d[0]));
    const float w1 = vmul(l1, a1), w2 = vmul(l2, a2), w3 = vmul(l3, a3);
    D[0] = vadd(w1, w3);
    D[1] = vadd(vmul(w1, vsub(u, c)), vmul(w3, vadd(u, c)));
    D[2] = vadd(vadd(vmul(w1, v), w2), vmul(w3, v));
  } else {
    const float g1 = phys - 1.f;
    const float a3 = vsub(d[2], vmul(v, d[0]));
    const float dE = vsub(d[3], vmul(a3, v));
    const float a2 = vmul(vmul(g1, vrcp(vmul(c, c))),
                          vsub(vadd(vmul(d[0], vsub(H, vmul(u, u))), vmul(u, d[1])), dE));
    const float a1 = vmul(vsub(vsub(vmul(d[0], vadd(u, c)), d[1]), vmul(c, a2)), r2c);
    const float a4 = vsub(d[0], vadd(a1, a2));
    const float w1 = vmul(l1, a1), w2 = vmul(l2, a2), w3 = vmul(l2, a3), w4 = vmul(l3, a4);
    const float k2 = vmul(0.5f, vfma(u, u, vmul(v, v)));
    D[0] = vadd(vadd(w1, w2), w4);
    D[1] = vadd(vadd(vmul(w1, vsub(u, c)), vmul(w2, u)), vmul(w4, vadd(u, c)));
    D[2] = vadd(vadd(vadd(vmul(w1, v), vmul(w2, v)), w3), vmul(w4, v));
    D[3] = vadd(vadd(vadd(vmul(w1, vsub(H, vmul(u, c))), vmul(w2, k2)), vmul(w3, v)),
                vmul(w4, vfma(u, c, H)));
  }
#pragma unroll
  for (int k = 0; k < C; ++k) F[k] = vsub(vmul(0.5f, vadd(FL[k], FR[k])), vmul(0.5f, D[k]));
}

// HLL formula with given speeds, three branches (Eq. 2.15 form)
template <int C>
__device__ __forceinline__ void hll_branches(const float (&L)[C], const float (&R)[C], const float (&FL)[C],
                                             const float (&FR)[C], float sL, float sR, float (&F)[C]) {
  if (sL >= 0.f) {
#pragma unroll
    for (int k = 0; k < C; ++k) F[k] = FL[k];
  } else if (sR < 0.f) {
#pragma unroll
    for (int k = 0; k < C; ++k) F[k] = FR[k];
  } else {
    const float r = vrcp(vsub(sR, sL));
#pragma unroll
    for (int k = 0; k < C; ++k)
      F[k] = vmul(vadd(vsub(vmul(sR, FL[k]), vmul(sL, FR[k])), vmul(vmul(sL, sR), vsub(R[k], L[k]))), r);
  }
}

// Q_*K = rho_K (s_K - u_K) / (s_K - s_*) [1, s_*, v_K, E_*] (Euler, Toro) or
// h_K (s_K - u_K) / (s_K - s_*) [1, s_*, v_K] (SWE); F_*K = F_K + s_K (Q_*K - Q_K).
template <int C, int EQ>
__device__ __forceinline__ void hllc_star(const float (&Q)[C], const float (&FK)[C], float uK, float pK,
                                          float sK, float ss, float (&F)[C]) {
  const float fac = vmul(vmul(Q[0], vsub(sK, uK)), vrcp(vsub(sK, ss)));
  float S[C];
  S[0] = fac;
  S[1] = vmul(fac, ss);
  S[2] = vmul(fac, vmul(Q[2], vrcp(Q[0])));
  if constexpr (EQ == EULER) {
    const float e = vadd(vmul(Q[3], vrcp(Q[0])),
                         vmul(vsub(ss, uK), vadd(ss, vmul(pK, vrcp(vmul(Q[0], vsub(sK, uK)))))));
    S[3] = vmul(fac, e);
  }
#pragma unroll
  for (int k = 0; k < C; ++k) F[k] = vadd(FK[k], vmul(sK, vsub(S[k], Q[k])));
}

// Numerical flux `flux` (not HLL) of two face-frame states; `nu` is the
// Lax-Friedrichs viscosity of this face's direction.
template <int C, int EQ>
__device__ __forceinline__ void scheme_flux(int flux, const float (&L)[C], const float (&R)[C], float phys,
                                            float nu, float (&F)[C]) {
  float FL[C], FR[C], uL, cL, pL, uR, cR, pR;
  frame_state<C, EQ>(L, phys, FL, uL, cL, pL);
  frame_state<C, EQ>(R, phys, FR, uR, cR, pR);
  if (flux == FLUX_LF) {
    central<C>(FL, FR, L, R, nu, F);
  } else if (flux == FLUX_RUSANOV) {
    const float s = vmul(0.5f, fmaxf(vadd(fabsf(uL), cL), vadd(fabsf(uR), cR)));
    central<C>(FL, FR, L, R, s, F);
  } else if (flux == FLUX_ROE) {
    roe_flux<C, EQ>(L, R, FL, FR, pL, pR, phys, F);
  } else if (flux == FLUX_HLLE) {
    float u, v, c, H;
    roe_state<C, EQ>(L, R, phys, u, v, c, H, pL, pR);
    const float sL = fminf(fminf(vsub(uL, cL), vsub(u, c)), 0.f);
    const float sR = fmaxf(fmaxf(vadd(uR, cR), vadd(u, c)), 0.f);
    hll_branches<C>(L, R, FL, FR, sL, sR, F);
  } else {   // HLLC
    const float sL = fminf(vsub(uL, cL), vsub(uR, cR));
    const float sR = fmaxf(vadd(uL, cL), vadd(uR, cR));
    float num, den;
    if constexpr (EQ == SWE) {
      num = vsub(vmul(vmul(sL, R[0]), vsub(uR, sR)), vmul(vmul(sR, L[0]), vsub(uL, sL)));
      den = vsub(vmul(R[0], vsub(uR, sR)), vmul(L[0], vsub(uL, sL)));
    } else {
      num = vsub(vadd(vsub(pR, pL), vmul(vmul(L[0], uL), vsub(sL, uL))), vmul(vmul(R[0], uR), vsub(sR, uR)));
      den = vsub(vmul(L[0], vsub(sL, uL)), vmul(R[0], vsub(sR, uR)));
    }
    const float ss = vmul(num, vrcp(den));
    if (sL >= 0.f) {
#pragma unroll
      for (int k = 0; k < C; ++k) F[k] = FL[k];
    } else if (ss >= 0.f) {
      hllc_star<C, EQ>(L, FL, uL, pL, sL, ss, F);
    } else if (sR > 0.f) {
      hllc_star<C, EQ>(R, FR, uR, pR, sR, ss, F);
    } else {
#pragma unroll
      for (int k = 0; k < C; ++k) F[k] = FR[k];
    }
  }
}

}  // namespace fvk
