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

enum Eq { SWE = 0, EULER = 1 };

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
  unsigned done;       // 1 once t reached t_end (or REPLAY ran out): stages skip all work
  unsigned exhausted;  // REPLAY has no dt left for the next step
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

// Eq. 2.18 limiter on undivided differences: a if |a| < |b|, b if
// |b| <= |a|, and 0 unless ab > 0.
__device__ __forceinline__ float minmod(float a, float b) {
  float r = fabsf(a) < fabsf(b) ? a : b;
  return (a * b > 0.f) ? r : 0.f;
}

// HLL flux (Eq. 2.15) of two face-frame SWE states (h, m_normal, m_tangential).
// Davis wave-speed estimates s_L = min(u_L - c_L, u_R - c_R),
// s_R = max(u_L + c_L, u_R + c_R).
__device__ __forceinline__ void hll_swe(float hL, float mL, float tL, float hR, float mR,
                                        float tR, float g, float& F0, float& F1, float& F2) {
  const float uL = mL / hL, uR = mR / hR;
  const float cL = sqrtf(g * hL), cR = sqrtf(g * hR);
  const float sL = fminf(uL - cL, uR - cR);
  const float sR = fmaxf(uL + cL, uR + cR);
  const float FL0 = mL, FL1 = mL * uL + 0.5f * g * hL * hL, FL2 = tL * uL;
  const float FR0 = mR, FR1 = mR * uR + 0.5f * g * hR * hR, FR2 = tR * uR;
  if (sL >= 0.f) {
    F0 = FL0; F1 = FL1; F2 = FL2;
  } else if (sR < 0.f) {
    F0 = FR0; F1 = FR1; F2 = FR2;
  } else {
    const float inv = 1.f / (sR - sL);
    const float ss = sL * sR;
    F0 = (sR * FL0 - sL * FR0 + ss * (hR - hL)) * inv;
    F1 = (sR * FL1 - sL * FR1 + ss * (mR - mL)) * inv;
    F2 = (sR * FL2 - sL * FR2 + ss * (tR - tL)) * inv;
  }
}

// HLL flux of two face-frame Euler states (rho, m_normal, m_tangential, E);
// ideal gas p = (gamma - 1)(E - (m^2 + t^2) / (2 rho)), c = sqrt(gamma p / rho).
__device__ __forceinline__ void hll_euler(const float* L, const float* R, float gamma,
                                          float* F) {
  const float uL = L[1] / L[0], vL = L[2] / L[0];
  const float uR = R[1] / R[0], vR = R[2] / R[0];
  const float pL = (gamma - 1.f) * (L[3] - 0.5f * (L[1] * uL + L[2] * vL));
  const float pR = (gamma - 1.f) * (R[3] - 0.5f * (R[1] * uR + R[2] * vR));
  const float cL = sqrtf(gamma * pL / L[0]), cR = sqrtf(gamma * pR / R[0]);
  const float sL = fminf(uL - cL, uR - cR);
  const float sR = fmaxf(uL + cL, uR + cR);
  const float FL[4] = {L[1], L[1] * uL + pL, L[2] * uL, uL * (L[3] + pL)};
  const float FR[4] = {R[1], R[1] * uR + pR, R[2] * uR, uR * (R[3] + pR)};
  if (sL >= 0.f) {
#pragma unroll
    for (int c = 0; c < 4; ++c) F[c] = FL[c];
  } else if (sR < 0.f) {
#pragma unroll
    for (int c = 0; c < 4; ++c) F[c] = FR[c];
  } else {
    const float inv = 1.f / (sR - sL);
    const float ss = sL * sR;
#pragma unroll
    for (int c = 0; c < 4; ++c) F[c] = (sR * FL[c] - sL * FR[c] + ss * (R[c] - L[c])) * inv;
  }
}

// Courant rate of one cell, (|u| + c)/dx + (|v| + c)/dy: the 2D Courant
// number of the unsplit update is dt times its maximum (Eq. 2.10 summed over
// the two directions).  Also the cell's health bits.
__device__ __forceinline__ float cell_rate_swe(float h, float hu, float hv, float g, float rdx,
                                               float rdy, unsigned& bad) {
  const float u = hu / h, v = hv / h;
  const float c = sqrtf(g * h);
  const float a = (fabsf(u) + c) * rdx + (fabsf(v) + c) * rdy;
  if (!(h > 0.f)) bad |= FV_HEALTH_NONPOSITIVE;
  if (!isfinite(h) || !isfinite(hu) || !isfinite(hv)) bad |= FV_HEALTH_NONFINITE;
  return a;
}

__device__ __forceinline__ float cell_rate_euler(const float* q, float gamma, float rdx,
                                                 float rdy, unsigned& bad) {
  const float u = q[1] / q[0], v = q[2] / q[0];
  const float p = (gamma - 1.f) * (q[3] - 0.5f * (q[1] * u + q[2] * v));
  const float c = sqrtf(gamma * p / q[0]);
  const float a = (fabsf(u) + c) * rdx + (fabsf(v) + c) * rdy;
  if (!(q[0] > 0.f) || !(p > 0.f)) bad |= FV_HEALTH_NONPOSITIVE;
  if (!isfinite(q[0]) || !isfinite(q[1]) || !isfinite(q[2]) || !isfinite(q[3]))
    bad |= FV_HEALTH_NONFINITE;
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
  c->done = c->exhausted;
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
