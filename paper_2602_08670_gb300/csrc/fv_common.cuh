// fv_common.cuh — definitions shared by the CUDA translation units of libfv.
//
// Device-side physics of the finite-volume step: MINMOD (Eq. 2.18), the
// shallow-water and Euler fluxes in a face-normal frame (Eqs. 2.3-2.5, 2.24),
// the HLL flux (Eq. 2.15), and the per-member control block that carries the
// CFL time step (Eq. 2.10), the simulated time and the health word between
// kernel launches without host round trips.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/fv.h"

namespace fvk {

enum Eq { SWE = 0, EULER = 1, SPHERE = 2 };   // SPHERE: shallow water on the sphere, C = 4

// ---------------------------------------------------------------------------
// Per-member control block (device memory, one per batch member)
// ---------------------------------------------------------------------------
struct Ctrl {
  double t;            // simulated time reached by the completed steps
  double dt;           // dt of the step in progress / next step
  double t_end;        // stop time (<= 0: none)
  double amax_last;    // max Courant rate (|u|+c)/dx + (|v|+c)/dy of the last state
  long long step;      // completed steps
  unsigned amax_bits;  // running max Courant rate of the state being produced (float bits)
  unsigned blocks_done;// blocks of the current reduction that have finished
  unsigned health;     // FV_HEALTH_* bits
  unsigned done;       // 1 once t reached t_end, step reached step_end or REPLAY ran out: stages skip all work
  unsigned exhausted;  // REPLAY has no dt left for the next step
  long long step_end;  // stop once this many steps are complete (<= 0: no limit)
};

// Parameters of the time-step rule, shared by all members (device memory).
struct DtParams {
  int mode;            // FV_DT_*
  int replay_len;
  double cfl;          // target 2D Courant number
  double dt_fixed;
  const double* replay;
};

// ---------------------------------------------------------------------------
// Physics helpers
// ---------------------------------------------------------------------------

// Arithmetic of the step, written once for scalars (float) and for pairs of
// cells (float2).  The float2 forms use the packed FP32 instructions of sm_100+
// (fma/add/sub/mul .rn.f32x2), whose per-component result is that of the
// scalar __fmaf_rn / __fadd_rn / __fmul_rn; the library is compiled without
// implicit FMA contraction.  So a face or a cell gives bitwise the
// same result in every kernel, packed or not, and in both directions (x faces
// and rotated y faces).

// Scalar ops as PTX with explicit rounding as well, so that the compiler
// cannot substitute another instruction sequence on one side only.
__device__ __forceinline__ float vadd(float a, float b) {
  float d;
  asm("add.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float vsub(float a, float b) {
  float d;
  asm("sub.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float vmul(float a, float b) {
  float d;
  asm("mul.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float vfma(float a, float b, float c) {
  float d;
  asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ float vneg(float a) { return -a; }
// 1/x and sqrt(x) through the SFU approximations (rcp.approx, sqrt.approx:
// a few ulp, well inside the FP32 roundoff of the step).  Arguments are depths, densities, pressures and wave-speed sums:
// normal positive numbers.
__device__ __forceinline__ float vrcp(float x) {
  float d;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(d) : "f"(x));
  return d;
}
__device__ __forceinline__ float vsqrt(float x) {
  float d;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(d) : "f"(x));
  return d;
}
template <class V> __device__ __forceinline__ V vsplat(float x);
template <> __device__ __forceinline__ float vsplat<float>(float x) { return x; }

// Packed ops as PTX with an explicit rounding mode: such instructions are
// never contracted, so a packed multiply followed by a packed add stays two
// roundings, exactly like the scalar __fmul_rn / __fadd_rn pair.
__device__ __forceinline__ unsigned long long pk2(float2 v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ float2 vadd(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(d);
}
__device__ __forceinline__ float2 vmin(float2 a, float2 b) {
  return make_float2(fminf(a.x, b.x), fminf(a.y, b.y));
}
__device__ __forceinline__ float2 vmax(float2 a, float2 b) {
  return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y));
}
__device__ __forceinline__ float2 vabs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 vrcp(float2 x) { return make_float2(vrcp(x.x), vrcp(x.y)); }
__device__ __forceinline__ float2 vsqrt(float2 x) { return make_float2(vsqrt(x.x), vsqrt(x.y)); }
template <> __device__ __forceinline__ float2 vsplat<float2>(float x) { return make_float2(x, x); }

// Eq. 2.18 limiter on undivided differences: a if |a| < |b|, b if
// |b| <= |a|, and 0 unless ab > 0 -- i.e. the median of (a, b, 0).
__device__ __forceinline__ float minmod(float a, float b) {
  return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.f));
}
__device__ __forceinline__ float2 minmod(float2 a, float2 b) {
  return make_float2(minmod(a.x, b.x), minmod(a.y, b.y));
}

// Face states from the minmod slopes of the two cells next to the face:
// Q^L = Q_i + s_i / 2, Q^R = Q_{i+1} - s_{i+1} / 2.
template <class V>
__device__ __forceinline__ V face_left(V q, V slope) { return vfma(vsplat<V>(0.5f), slope, q); }
template <class V>
__device__ __forceinline__ V face_right(V q, V slope) { return vfma(vsplat<V>(-0.5f), slope, q); }

// HLL weights of Eq. 2.15 in branch-free form.  With s_L' = min(s_L, 0) and
// s_R' = max(s_R, 0) the three branches become one expression,
//   F = a FL + b FR + g (qR - qL),
//   a = s_R' / (s_R' - s_L'), b = -s_L' / (s_R' - s_L'), g = s_L' s_R' / (s_R' - s_L'),
// which equals F_L when 0 <= s_L, F_R when s_R < 0 and the HLL flux between
// (identical in exact arithmetic, to rounding in floating point).
template <class V>
struct HllW {
  V a, b, g;
};
template <class V>
__device__ __forceinline__ HllW<V> hll_weights(V sL, V sR) {
  const V zL = vmin(sL, vsplat<V>(0.f)), zR = vmax(sR, vsplat<V>(0.f));
  const V inv = vrcp(vsub(zR, zL));
  HllW<V> w;
  w.a = vmul(zR, inv);
  w.b = vneg(vmul(zL, inv));
  w.g = vmul(vmul(zL, zR), inv);
  return w;
}
template <class V>
__device__ __forceinline__ V hll_mix(const HllW<V>& w, V FL, V FR, V qL, V qR) {
  return vfma(w.g, vsub(qR, qL), vfma(w.b, FR, vmul(w.a, FL)));
}

// HLL flux (Eq. 2.15) of two face-frame SWE states (h, m_normal, m_tangential).
// Davis wave-speed estimates s_L = min(u_L - c_L, u_R - c_R),
// s_R = max(u_L + c_L, u_R + c_R), c = sqrt(g h).
template <class V>
__device__ __forceinline__ void hll_swe(V hL, V mL, V tL, V hR, V mR, V tR, float g, V& F0, V& F1,
                                        V& F2) {
  const V gv = vsplat<V>(g), half = vsplat<V>(0.5f);
  const V uL = vmul(mL, vrcp(hL)), uR = vmul(mR, vrcp(hR));
  const V ghL = vmul(gv, hL), ghR = vmul(gv, hR);
  const V cL = vsqrt(ghL), cR = vsqrt(ghR);
  const V sL = vmin(vsub(uL, cL), vsub(uR, cR));
  const V sR = vmax(vadd(uL, cL), vadd(uR, cR));
  const HllW<V> w = hll_weights(sL, sR);
  F0 = hll_mix(w, mL, mR, hL, hR);
  const V FL1 = vfma(mL, uL, vmul(vmul(half, ghL), hL));
  const V FR1 = vfma(mR, uR, vmul(vmul(half, ghR), hR));
  F1 = hll_mix(w, FL1, FR1, mL, mR);
  F2 = hll_mix(w, vmul(tL, uL), vmul(tR, uR), tL, tR);
}

// HLL flux of two face-frame Euler states (rho, m_normal, m_tangential, E);
// ideal gas p = (gamma - 1)(E - (m^2 + t^2) / (2 rho)), c = sqrt(gamma p / rho).
template <class V>
__device__ __forceinline__ void hll_euler(const V* L, const V* R, float gamma, V* F) {
  const V gm1 = vsplat<V>(gamma - 1.f), gv = vsplat<V>(gamma), mhalf = vsplat<V>(-0.5f);
  const V rL = vrcp(L[0]), rR = vrcp(R[0]);
  const V uL = vmul(L[1], rL), vL = vmul(L[2], rL);
  const V uR = vmul(R[1], rR), vR = vmul(R[2], rR);
  const V pL = vmul(gm1, vfma(mhalf, vfma(L[1], uL, vmul(L[2], vL)), L[3]));
  const V pR = vmul(gm1, vfma(mhalf, vfma(R[1], uR, vmul(R[2], vR)), R[3]));
  const V cL = vsqrt(vmul(vmul(gv, pL), rL)), cR = vsqrt(vmul(vmul(gv, pR), rR));
  const V sL = vmin(vsub(uL, cL), vsub(uR, cR));
  const V sR = vmax(vadd(uL, cL), vadd(uR, cR));
  const HllW<V> w = hll_weights(sL, sR);
  F[0] = hll_mix(w, L[1], R[1], L[0], R[0]);
  F[1] = hll_mix(w, vfma(L[1], uL, pL), vfma(R[1], uR, pR), L[1], R[1]);
  F[2] = hll_mix(w, vmul(L[2], uL), vmul(R[2], uR), L[2], R[2]);
  F[3] = hll_mix(w, vmul(uL, vadd(L[3], pL)), vmul(uR, vadd(R[3], pR)), L[3], R[3]);
}

// Flux divergence of one cell, -(F_e - F_w)/dx - (G_n - G_s)/dy (Eqs. 2.9,
// 2.23); symmetric in x and y.
template <class V>
__device__ __forceinline__ V divergence(V Fw, V Fe, V Gs, V Gn, float rdx, float rdy) {
  return vneg(vadd(vmul(vsub(Fe, Fw), vsplat<V>(rdx)), vmul(vsub(Gn, Gs), vsplat<V>(rdy))));
}

// SSP-RK2 (Eq. 2.19).  Stage 1: q + dt L.  Stage 2: qn/2 + q1/2 + (dt/2) L.
template <class V>
__device__ __forceinline__ V rk_stage1(V q, float dt, V L) { return vfma(vsplat<V>(dt), L, q); }
template <class V>
__device__ __forceinline__ V rk_stage2(V qn, V q1, float hdt, V L) {
  const V half = vsplat<V>(0.5f);
  return vfma(vsplat<V>(hdt), L, vadd(vmul(half, qn), vmul(half, q1)));
}

// Courant rate of one cell, (|u| + c)/dx + (|v| + c)/dy: the 2D Courant
// number of the unsplit update is dt times its maximum (Eq. 2.10 summed over
// the two directions).  Health bits: a non-positive depth/density/pressure or
// a non-finite rate (any NaN/Inf in the state) flag the cell.
__device__ __forceinline__ float cell_rate_swe(float h, float hu, float hv, float g, float rdx,
                                               float rdy, unsigned& bad) {
  const float r = vrcp(h);
  const float c = vsqrt(vmul(g, h));
  const float a = vfma(vadd(fabsf(vmul(hu, r)), c), rdx, vmul(vadd(fabsf(vmul(hv, r)), c), rdy));
  bad |= (h > 0.f) ? 0u : (unsigned)FV_HEALTH_NONPOSITIVE;
  bad |= (a < INFINITY) ? 0u : (unsigned)FV_HEALTH_NONFINITE;
  return a;
}

__device__ __forceinline__ float cell_rate_euler(const float* q, float gamma, float rdx,
                                                 float rdy, unsigned& bad) {
  const float r = vrcp(q[0]);
  const float u = vmul(q[1], r), v = vmul(q[2], r);
  const float p = vmul(gamma - 1.f, vfma(-0.5f, vfma(q[1], u, vmul(q[2], v)), q[3]));
  const float c = vsqrt(vmul(vmul(gamma, p), r));
  const float a = vfma(vadd(fabsf(u), c), rdx, vmul(vadd(fabsf(v), c), rdy));
  bad |= (q[0] > 0.f && p > 0.f) ? 0u : (unsigned)FV_HEALTH_NONPOSITIVE;
  bad |= (a < INFINITY) ? 0u : (unsigned)FV_HEALTH_NONFINITE;
  return a;
}

// True if the member's work is finished; a stage attempted after REPLAY ran
// out of dt values raises FV_HEALTH_REPLAY_END.  Uniform per block.
__device__ __forceinline__ bool skip_if_done(Ctrl* c) {
  if (!c->done) return false;
  if (c->exhausted && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    atomicOr(&c->health, FV_HEALTH_REPLAY_END);
  return true;
}

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Block-wide max of a non-negative float (NaN ignored) and OR of health bits;
// the result is valid in thread 0.  `red` needs 2 * (blockDim / 32) words.
__device__ __forceinline__ void block_reduce_max_or(float& m, unsigned& bad, unsigned* red) {
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[warp] = __float_as_uint(m);
    red[nw + warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      m = fmaxf(m, __uint_as_float(red[w]));
      bad |= red[nw + w];
    }
  }
}

// Called by thread 0 of a block after its reduction: publish the block's max
// Courant rate and health bits; the last block of the member's grid closes the
// step (advance t, choose the next dt by Eq. 2.10 or the FIXED/REPLAY rule,
// apply t_end) and resets the reduction.  `advance` is false for the initial
// reduction at state creation.
__device__ inline void publish_and_close(Ctrl* c, const DtParams* dp, float m, unsigned bad,
                                         unsigned nblocks, bool advance) {
  if (bad) atomicOr(&c->health, bad);
  atomicMax(&c->amax_bits, __float_as_uint(m));
  __threadfence();
  const unsigned prev = atomicAdd(&c->blocks_done, 1u);
  if (prev != nblocks - 1) return;
  __threadfence();
  const float amax = __uint_as_float(atomicAdd(&c->amax_bits, 0u));
  if (advance) {
    c->t += c->dt;
    c->step += 1;
  }
  double dt;
  if (dp->mode == FV_DT_ADAPTIVE) {
    dt = dp->cfl / (double)amax;
  } else if (dp->mode == FV_DT_FIXED) {
    dt = dp->dt_fixed;
  } else {
    if (c->step < dp->replay_len) {
      dt = dp->replay[c->step];
      c->exhausted = 0u;
    } else {
      dt = 0.0;
      c->exhausted = 1u;   // flagged only if a step is attempted (skip_if_done)
    }
  }
  if (dp->mode != FV_DT_ADAPTIVE && (double)amax * dt > 1.0) c->health |= FV_HEALTH_CFL;
  c->done = c->exhausted | (c->step_end > 0 && c->step >= c->step_end ? 1u : 0u);
  if (c->t_end > 0.0) {
    const double rem = c->t_end - c->t;
    if (rem <= 0.0) {
      dt = 0.0;
      c->done = 1u;
    } else if (dt > rem) {
      dt = rem;
    }
  }
  c->dt = dt;
  c->amax_last = amax;
  c->amax_bits = 0u;
  __threadfence();
  c->blocks_done = 0u;
}

}  // namespace fvk

// ---------------------------------------------------------------------------
// Host-side helpers shared by the API translation units
// ---------------------------------------------------------------------------
namespace fvh {
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
}  // namespace fvh

#define FV_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return fvh::cuda_fail(_e, #expr); \
  } while (0)
