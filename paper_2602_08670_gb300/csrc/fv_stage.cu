// fv_stage.cu — fused SSP-RK2 stage kernels of the plain finite-volume step.
//
// One launch = one Runge-Kutta stage of Eq. 2.19 over every member:
//   load the stage input tile with a 2-cell periodic halo into shared memory,
//   reconstruct face states by MUSCL-minmod (Eq. 2.18),
//   compute HLL fluxes (Eq. 2.15) on x faces and on y faces (the latter in
//   the rotated frame of Eq. 2.24: normal momentum = hv),
//   form the flux divergence (Eqs. 2.9 / 2.23) and the RK combine,
//   and, in stage 2, reduce the Courant rate (|u|+c)/dx + (|v|+c)/dy of the
//   new state by warp shuffles for the next CFL time step (Eq. 2.10).
// Face values and fluxes live in shared memory only; HBM sees the stage input
// (plus halo re-reads that hit L2), q^n in stage 2, and the stage output.
#include <cuda_runtime.h>

#include "fv_common.cuh"
#include "fv_kernels.h"

namespace fvk {

namespace {

constexpr int TX = 64;           // tile width (cells)
constexpr int TY = 16;           // tile height (cells)
constexpr int SX = TX + 4;       // staged width incl. 2-cell halo each side
constexpr int SY = TY + 4;
constexpr int NT = 256;          // threads per block

template <int C>
constexpr int stage_smem_bytes() {
  return (C * (SY * SX + TY * (TX + 1) + (TY + 1) * TX) + 4 * (NT / 32)) * 4;
}

struct StageArgs {
  const float* qin;
  const float* qn;
  float* qout;
  Ctrl* ctrl;
  const DtParams* dp;
  int nx, ny;
  long long plane, member;
  float rdx, rdy, phys;
};

// Normal-frame flux of one face from its four-cell stencil.  `rot` selects the
// y-face frame (normal momentum = component 2).
template <int C, int EQ>
__device__ __forceinline__ void stencil_flux(const float (&m)[C], const float (&a)[C],
                                             const float (&b)[C], const float (&p)[C], bool rot,
                                             float phys, float (&F)[C]) {
  float L[C], R[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    L[c] = a[c] + 0.5f * minmod(a[c] - m[c], b[c] - a[c]);
    R[c] = b[c] - 0.5f * minmod(b[c] - a[c], p[c] - b[c]);
  }
  if (rot) {
    float t = L[1]; L[1] = L[2]; L[2] = t;
    t = R[1]; R[1] = R[2]; R[2] = t;
  }
  if constexpr (EQ == SWE) {
    hll_swe(L[0], L[1], L[2], R[0], R[1], R[2], phys, F[0], F[1], F[2]);
  } else {
    hll_euler(L, R, phys, F);
  }
  if (rot) {
    float t = F[1]; F[1] = F[2]; F[2] = t;
  }
}

template <int C, int EQ, int STAGE>
__global__ void __launch_bounds__(NT) stage_minmod_kernel(StageArgs a) {
  extern __shared__ float smem[];
  float* sq = smem;                          // [C][SY][SX]
  float* sF = sq + C * SY * SX;              // [C][TY][TX+1]
  float* sG = sF + C * TY * (TX + 1);        // [C][TY+1][TX]
  unsigned* red = reinterpret_cast<unsigned*>(sG + C * (TY + 1) * TX);

  const int b = blockIdx.z;
  Ctrl* ctrl = a.ctrl + b;
  if (skip_if_done(ctrl)) return;
  const float dt = (float)ctrl->dt;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const float* qin = a.qin + b * a.member;
  const int tid = threadIdx.x;

  // 1. stage the tile and its periodic halo
  for (int idx = tid; idx < C * SY * SX; idx += NT) {
    const int c = idx / (SY * SX);
    const int r = idx - c * (SY * SX);
    const int sy = r / SX, sx = r - sy * SX;
    const int gx = wrap(x0 - 2 + sx, a.nx), gy = wrap(y0 - 2 + sy, a.ny);
    sq[idx] = qin[c * a.plane + (long long)gy * a.nx + gx];
  }
  __syncthreads();

  // 2a. x faces: face k of tile row r lies between cells x0-1+k and x0+k
  for (int idx = tid; idx < TY * (TX + 1); idx += NT) {
    const int r = idx / (TX + 1), k = idx - r * (TX + 1);
    const float* row = sq + (r + 2) * SX + k;
    float m[C], s0[C], s1[C], p[C], F[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float* rc = row + c * SY * SX;
      m[c] = rc[0]; s0[c] = rc[1]; s1[c] = rc[2]; p[c] = rc[3];
    }
    stencil_flux<C, EQ>(m, s0, s1, p, false, a.phys, F);
#pragma unroll
    for (int c = 0; c < C; ++c) sF[(c * TY + r) * (TX + 1) + k] = F[c];
  }
  // 2b. y faces: face k of tile column i lies between rows y0-1+k and y0+k
  for (int idx = tid; idx < (TY + 1) * TX; idx += NT) {
    const int k = idx / TX, i = idx - k * TX;
    const float* col = sq + k * SX + (i + 2);
    float m[C], s0[C], s1[C], p[C], F[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float* cc = col + c * SY * SX;
      m[c] = cc[0]; s0[c] = cc[SX]; s1[c] = cc[2 * SX]; p[c] = cc[3 * SX];
    }
    stencil_flux<C, EQ>(m, s0, s1, p, true, a.phys, F);
#pragma unroll
    for (int c = 0; c < C; ++c) sG[(c * (TY + 1) + k) * TX + i] = F[c];
  }
  __syncthreads();

  // 3. divergence and RK combine
  float amax = 0.f;
  unsigned bad = 0u;
  const float* qn = a.qn + b * a.member;
  float* qout = a.qout + b * a.member;
  for (int idx = tid; idx < TY * TX; idx += NT) {
    const int r = idx / TX, i = idx - r * TX;
    const int gx = x0 + i, gy = y0 + r;
    if (gx >= a.nx || gy >= a.ny) continue;
    const long long off = (long long)gy * a.nx + gx;
    float out[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float Fw = sF[(c * TY + r) * (TX + 1) + i];
      const float Fe = sF[(c * TY + r) * (TX + 1) + i + 1];
      const float Gs = sG[(c * (TY + 1) + r) * TX + i];
      const float Gn = sG[(c * (TY + 1) + r + 1) * TX + i];
      // products rounded separately (no FMA contraction) so that x and y
      // enter symmetrically: a transposed state gives the transposed result
      const float L = -__fadd_rn(__fmul_rn(Fe - Fw, a.rdx), __fmul_rn(Gn - Gs, a.rdy));
      const float q = sq[(c * SY + r + 2) * SX + i + 2];
      if (STAGE == 1) {
        out[c] = q + dt * L;
      } else {
        out[c] = 0.5f * qn[c * a.plane + off] + 0.5f * q + 0.5f * dt * L;
      }
      qout[c * a.plane + off] = out[c];
    }
    if (STAGE == 2) {
      float s;
      if constexpr (EQ == SWE) {
        s = cell_rate_swe(out[0], out[1], out[2], a.phys, a.rdx, a.rdy, bad);
      } else {
        s = cell_rate_euler(out, a.phys, a.rdx, a.rdy, bad);
      }
      amax = fmaxf(amax, s);
    }
  }
  if (STAGE == 2) {
    block_reduce_max_or(amax, bad, red);
    if (tid == 0) publish_and_close(ctrl, a.dp, amax, bad, gridDim.x * gridDim.y, true);
  }
}

template <int C, int EQ>
__global__ void __launch_bounds__(256) wavespeed_init_kernel(const float* q, Ctrl* ctrl,
                                                             const DtParams* dp, int nx, int ny,
                                                             long long plane, long long member,
                                                             float phys, float rdx, float rdy) {
  __shared__ unsigned red[16];
  const int b = blockIdx.y;
  const float* qb = q + b * member;
  float amax = 0.f;
  unsigned bad = 0u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
       i += (long long)gridDim.x * blockDim.x) {
    float v[C];
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = qb[c * plane + i];
    float s;
    if constexpr (EQ == SWE) {
      s = cell_rate_swe(v[0], v[1], v[2], phys, rdx, rdy, bad);
    } else {
      s = cell_rate_euler(v, phys, rdx, rdy, bad);
    }
    amax = fmaxf(amax, s);
  }
  block_reduce_max_or(amax, bad, red);
  if (threadIdx.x == 0) publish_and_close(ctrl + b, dp, amax, bad, gridDim.x, false);
}

// Deterministic FP64 sums: each block writes its partial sums (fixed
// assignment of cells to blocks and a fixed tree), then one block per
// member adds the partials in index order.
constexpr int DIAG_BLOCKS = 256;
constexpr int DIAG_NT = 256;

template <int C, int EQ>
__global__ void __launch_bounds__(DIAG_NT) diag_partial_kernel(const float* q, double* partials,
                                                               long long plane, long long member,
                                                               double phys) {
  __shared__ double sh[DIAG_NT];
  const int b = blockIdx.y;
  const float* qb = q + b * member;
  double acc[C + 1];
#pragma unroll
  for (int c = 0; c <= C; ++c) acc[c] = 0.0;
  for (long long i = blockIdx.x * (long long)DIAG_NT + threadIdx.x; i < plane;
       i += (long long)DIAG_BLOCKS * DIAG_NT) {
    double v[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      v[c] = (double)qb[c * plane + i];
      acc[c] += v[c];
    }
    if constexpr (EQ == SWE) {
      const double u = v[1] / v[0], w = v[2] / v[0];
      acc[C] += 0.5 * phys * v[0] * v[0] + 0.5 * (u * u + w * w) * v[0];
    } else {
      const double u = v[1] / v[0], w = v[2] / v[0];
      acc[C] += 0.5 * v[0] * (u * u + w * w);
    }
  }
  for (int c = 0; c <= C; ++c) {
    sh[threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = DIAG_NT / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[((long long)b * (C + 1) + c) * DIAG_BLOCKS + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

__global__ void diag_final_kernel(const double* partials, double* out, int C1, double area) {
  const int b = blockIdx.x;
  for (int c = threadIdx.x; c < C1; c += blockDim.x) {
    double s = 0.0;
    const double* p = partials + ((long long)b * C1 + c) * DIAG_BLOCKS;
    for (int k = 0; k < DIAG_BLOCKS; ++k) s += p[k];
    out[b * C1 + c] = s * area;
  }
}

__global__ void set_t_end_kernel(Ctrl* ctrl, int B, double t_end) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  Ctrl* c = ctrl + b;
  c->t_end = t_end;
  c->done = c->exhausted;
  if (t_end > 0.0) {
    const double rem = t_end - c->t;
    if (rem <= 0.0) {
      c->done = 1u;
      c->dt = 0.0;
    } else if (c->dt > rem) {
      c->dt = rem;
    }
  }
}

template <int C, int EQ, int STAGE>
cudaError_t launch_stage_t(const Geom& g, const float* qin, const float* qn, float* qout,
                           Ctrl* ctrl, const DtParams* dp, cudaStream_t s) {
  constexpr int smem = stage_smem_bytes<C>();
  auto kern = stage_minmod_kernel<C, EQ, STAGE>;
  static bool attr_set = false;   // set once per process (per template instance)
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  StageArgs a{qin, qn, qout, ctrl, dp, g.nx, g.ny, g.plane(), g.member(),
              (float)(1.0 / g.dx), (float)(1.0 / g.dy), g.phys};
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, g.B);
  kern<<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stage_minmod(const Geom& g, int stage, const float* qin, const float* qn,
                                float* qout, Ctrl* ctrl, const DtParams* dp, cudaStream_t s) {
  if (g.eq == SWE) {
    return stage == 1 ? launch_stage_t<3, SWE, 1>(g, qin, qn, qout, ctrl, dp, s)
                      : launch_stage_t<3, SWE, 2>(g, qin, qn, qout, ctrl, dp, s);
  }
  return stage == 1 ? launch_stage_t<4, EULER, 1>(g, qin, qn, qout, ctrl, dp, s)
                    : launch_stage_t<4, EULER, 2>(g, qin, qn, qout, ctrl, dp, s);
}

cudaError_t launch_wavespeed_init(const Geom& g, const float* q, Ctrl* ctrl, const DtParams* dp,
                                  cudaStream_t s) {
  long long blocks = (g.plane() + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  dim3 grid((unsigned)blocks, g.B);
  if (g.eq == SWE) {
    wavespeed_init_kernel<3, SWE><<<grid, 256, 0, s>>>(q, ctrl, dp, g.nx, g.ny, g.plane(),
                                                       g.member(), g.phys, (float)(1.0 / g.dx),
                                                       (float)(1.0 / g.dy));
  } else {
    wavespeed_init_kernel<4, EULER><<<grid, 256, 0, s>>>(q, ctrl, dp, g.nx, g.ny, g.plane(),
                                                         g.member(), g.phys, (float)(1.0 / g.dx),
                                                         (float)(1.0 / g.dy));
  }
  return cudaGetLastError();
}

long long diag_partials_size(const Geom& g) { return (long long)g.B * (g.C + 1) * DIAG_BLOCKS; }

cudaError_t launch_diagnostics(const Geom& g, const float* q, double* partials, double* out,
                               cudaStream_t s) {
  dim3 grid(DIAG_BLOCKS, g.B);
  if (g.eq == SWE) {
    diag_partial_kernel<3, SWE><<<grid, DIAG_NT, 0, s>>>(q, partials, g.plane(), g.member(),
                                                         g.phys_d);
  } else {
    diag_partial_kernel<4, EULER><<<grid, DIAG_NT, 0, s>>>(q, partials, g.plane(), g.member(),
                                                           g.phys_d);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<g.B, 32, 0, s>>>(partials, out, g.C + 1, g.dx * g.dy);
  return cudaGetLastError();
}

cudaError_t launch_set_t_end(Ctrl* ctrl, int B, double t_end, cudaStream_t s) {
  set_t_end_kernel<<<(B + 127) / 128, 128, 0, s>>>(ctrl, B, t_end);
  return cudaGetLastError();
}

}  // namespace fvk
