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

// Per-lane select: c >= 0 ? a : b (packed pairs lane by lane).
__device__ __forceinline__ float vsel_ge0(float c, float a, float b) { return c >= 0.f ? a : b; }
__device__ __forceinline__ float2 vsel_ge0(float2 c, float2 a, float2 b) {
  return make_float2(c.x >= 0.f ? a.x : b.x, c.y >= 0.f ? a.y : b.y);
}
__device__ __forceinline__ float vsel_gt0(float c, float a, float b) { return c > 0.f ? a : b; }
__device__ __forceinline__ float2 vsel_gt0(float2 c, float2 a, float2 b) {
  return make_float2(c.x > 0.f ? a.x : b.x, c.y > 0.f ? a.y : b.y);
}

// Physical x flux, normal velocity and sound speed of one face-frame state
// (V = float, or float2 for two faces at once).
template <int C, int EQ, class V>
__device__ __forceinline__ void frame_state(const V (&q)[C], float phys, V (&F)[C], V& u, V& c, V& p) {
  const V r = vrcp(q[0]);
  u = vmul(q[1], r);
  if constexpr (EQ == SWE) {
    const V gh = vmul(vsplat<V>(phys), q[0]);
    c = vsqrt(gh);
    p = vmul(vmul(vsplat<V>(0.5f), gh), q[0]);
    F[0] = q[1];
    F[1] = vfma(q[1], u, p);
    F[2] = vmul(q[2], u);
  } else {
    const V v = vmul(q[2], r);
    p = vmul(vsplat<V>(phys - 1.f), vfma(vsplat<V>(-0.5f), vfma(q[1], u, vmul(q[2], v)), q[3]));
    c = vsqrt(vmul(vmul(vsplat<V>(phys), p), r));
    F[0] = q[1];
    F[1] = vfma(q[1], u, p);
    F[2] = vmul(q[2], u);
    F[3] = vmul(u, vadd(q[3], p));
  }
}

// 1/2 (F_L + F_R) - nu (Q_R - Q_L)
template <int C, class V>
__device__ __forceinline__ void central(const V (&FL)[C], const V (&FR)[C], const V (&L)[C], const V (&R)[C],
                                        V nu, V (&F)[C]) {
#pragma unroll
  for (int k = 0; k < C; ++k) F[k] = vsub(vmul(vsplat<V>(0.5f), vadd(FL[k], FR[k])), vmul(nu, vsub(R[k], L[k])));
}

// Roe-averaged u, v, c (and H for Euler) of two face-frame states.
template <int C, int EQ, class V>
__device__ __forceinline__ void roe_state(const V (&L)[C], const V (&R)[C], float phys, V& u, V& v, V& c, V& H,
                                          V pL, V pR) {
  const V sL = vsqrt(L[0]), sR = vsqrt(R[0]);
  const V w = vrcp(vadd(sL, sR));
  u = vmul(vadd(vmul(L[1], vrcp(sL)), vmul(R[1], vrcp(sR))), w);
  v = vmul(vadd(vmul(L[2], vrcp(sL)), vmul(R[2], vrcp(sR))), w);
  if constexpr (EQ == SWE) {
    c = vsqrt(vmul(vsplat<V>(phys), vmul(vsplat<V>(0.5f), vadd(L[0], R[0]))));
    H = vsplat<V>(0.f);
  } else {
    const V HL = vmul(vadd(L[3], pL), vrcp(L[0]));
    const V HR = vmul(vadd(R[3], pR), vrcp(R[0]));
    H = vmul(vadd(vmul(sL, HL), vmul(sR, HR)), w);
    c = vsqrt(vmul(vsplat<V>(phys - 1.f), vsub(H, vmul(vsplat<V>(0.5f), vfma(u, u, vmul(v, v))))));
  }
}

template <int C, int EQ, class V>
__device__ __forceinline__ void roe_flux(const V (&L)[C], const V (&R)[C], const V (&FL)[C], const V (&FR)[C],
                                         V pL, V pR, float phys, V (&F)[C]) {
  V u, v, c, H;
  roe_state<C, EQ, V>(L, R, phys, u, v, c, H, pL, pR);
  V d[C];
#pragma unroll
  for (int k = 0; k < C; ++k) d[k] = vsub(R[k], L[k]);
  const V l1 = vabs(vsub(u, c)), l2 = vabs(u), l3 = vabs(vadd(u, c));
  const V r2c = vrcp(vadd(c, c));
  V D[C];
  if constexpr (EQ == SWE) {
    const V a1 = vmul(vsub(vmul(vadd(u, c), d[0]), d[1]), r2c);
    const V a3 = vmul(vsub(d[1], vmul(vsub(u, c), d[0])), r2c);
    const V a2 = vsub(d[2], vmul(v, d[0]));
    const V w1 = vmul(l1, a1), w2 = vmul(l2, a2), w3 = vmul(l3, a3);
    D[0] = vadd(w1, w3);
    D[1] = vadd(vmul(w1, vsub(u, c)), vmul(w3, vadd(u, c)));
    D[2] = vadd(vadd(vmul(w1, v), w2), vmul(w3, v));
  } else {
    const V g1 = vsplat<V>(phys - 1.f);
    const V a3 = vsub(d[2], vmul(v, d[0]));
    const V dE = vsub(d[3], vmul(a3, v));
    const V a2 = vmul(vmul(g1, vrcp(vmul(c, c))), vsub(vadd(vmul(d[0], vsub(H, vmul(u, u))), vmul(u, d[1])), dE));
    const V a1 = vmul(vsub(vsub(vmul(d[0], vadd(u, c)), d[1]), vmul(c, a2)), r2c);
    const V a4 = vsub(d[0], vadd(a1, a2));
    const V w1 = vmul(l1, a1), w2 = vmul(l2, a2), w3 = vmul(l2, a3), w4 = vmul(l3, a4);
    const V k2 = vmul(vsplat<V>(0.5f), vfma(u, u, vmul(v, v)));
    D[0] = vadd(vadd(w1, w2), w4);
    D[1] = vadd(vadd(vmul(w1, vsub(u, c)), vmul(w2, u)), vmul(w4, vadd(u, c)));
    D[2] = vadd(vadd(vadd(vmul(w1, v), vmul(w2, v)), w3), vmul(w4, v));
    D[3] = vadd(vadd(vadd(vmul(w1, vsub(H, vmul(u, c))), vmul(w2, k2)), vmul(w3, v)), vmul(w4, vfma(u, c, H)));
  }
#pragma unroll
  for (int k = 0; k < C; ++k)
    F[k] = vsub(vmul(vsplat<V>(0.5f), vadd(FL[k], FR[k])), vmul(vsplat<V>(0.5f), D[k]));
}

// Q_*K = rho_K (s_K - u_K) / (s_K - s_*) [1, s_*, v_K, E_*] (Euler, Toro) or
// h_K (s_K - u_K) / (s_K - s_*) [1, s_*, v_K] (SWE); F_*K = F_K + s_K (Q_*K - Q_K).
template <int C, int EQ, class V>
__device__ __forceinline__ void hllc_star(const V (&Q)[C], const V (&FK)[C], V uK, V pK, V sK, V ss, V (&F)[C]) {
  const V fac = vmul(vmul(Q[0], vsub(sK, uK)), vrcp(vsub(sK, ss)));
  V S[C];
  S[0] = fac;
  S[1] = vmul(fac, ss);
  S[2] = vmul(fac, vmul(Q[2], vrcp(Q[0])));
  if constexpr (EQ == EULER) {
    const V e = vadd(vmul(Q[3], vrcp(Q[0])), vmul(vsub(ss, uK), vadd(ss, vmul(pK, vrcp(vmul(Q[0], vsub(sK, uK)))))));
    S[3] = vmul(fac, e);
  }
#pragma unroll
  for (int k = 0; k < C; ++k) F[k] = vadd(FK[k], vmul(sK, vsub(S[k], Q[k])));
}

// Numerical flux `flux` (not HLL) of two face-frame states, for one face
// (V = float) or two faces at once (V = float2); `nu` is the Lax-Friedrichs
// viscosity of this face's direction.  Branches on wave speeds are taken per
// lane as selects, so both forms give the same value for each face.
template <int C, int EQ, class V>
__device__ __forceinline__ void scheme_flux(int flux, const V (&L)[C], const V (&R)[C], float phys, float nu,
                                            V (&F)[C]) {
  V FL[C], FR[C], uL, cL, pL, uR, cR, pR;
  frame_state<C, EQ, V>(L, phys, FL, uL, cL, pL);
  frame_state<C, EQ, V>(R, phys, FR, uR, cR, pR);
  if (flux == FLUX_LF) {
    central<C, V>(FL, FR, L, R, vsplat<V>(nu), F);
  } else if (flux == FLUX_RUSANOV) {
    const V s = vmul(vsplat<V>(0.5f), vmax(vadd(vabs(uL), cL), vadd(vabs(uR), cR)));
    central<C, V>(FL, FR, L, R, s, F);
  } else if (flux == FLUX_ROE) {
    roe_flux<C, EQ, V>(L, R, FL, FR, pL, pR, phys, F);
  } else if (flux == FLUX_HLLE) {
    V u, v, c, H;
    roe_state<C, EQ, V>(L, R, phys, u, v, c, H, pL, pR);
    const V zero = vsplat<V>(0.f);
    const V sL = vmin(vmin(vsub(uL, cL), vsub(u, c)), zero);
    const V sR = vmax(vmax(vadd(uR, cR), vadd(u, c)), zero);
    // three branches of Eq. 2.15 with these speeds: F_L if s_L >= 0, F_R if
    // s_R < 0 (never: s_R >= 0), else the HLL average
    const V r = vrcp(vsub(sR, sL));
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const V mid = vmul(vadd(vsub(vmul(sR, FL[k]), vmul(sL, FR[k])), vmul(vmul(sL, sR), vsub(R[k], L[k]))), r);
      F[k] = vsel_ge0(sL, FL[k], mid);
    }
  } else {   // HLLC
    const V sL = vmin(vsub(uL, cL), vsub(uR, cR));
    const V sR = vmax(vadd(uL, cL), vadd(uR, cR));
    V num, den;
    if constexpr (EQ == SWE) {
      num = vsub(vmul(vmul(sL, R[0]), vsub(uR, sR)), vmul(vmul(sR, L[0]), vsub(uL, sL)));
      den = vsub(vmul(R[0], vsub(uR, sR)), vmul(L[0], vsub(uL, sL)));
    } else {
      num = vsub(vadd(vsub(pR, pL), vmul(vmul(L[0], uL), vsub(sL, uL))), vmul(vmul(R[0], uR), vsub(sR, uR)));
      den = vsub(vmul(L[0], vsub(sL, uL)), vmul(R[0], vsub(sR, uR)));
    }
    const V ss = vmul(num, vrcp(den));
    V FsL[C], FsR[C];
    hllc_star<C, EQ, V>(L, FL, uL, pL, sL, ss, FsL);
    hllc_star<C, EQ, V>(R, FR, uR, pR, sR, ss, FsR);
    // F_L if s_L >= 0, F*_L if s_* >= 0, F*_R if s_R > 0, else F_R
#pragma unroll
    for (int k = 0; k < C; ++k)
      F[k] = vsel_ge0(sL, FL[k], vsel_ge0(ss, FsL[k], vsel_gt0(sR, FsR[k], FR[k])));
  }
}

}  // namespace fvk
