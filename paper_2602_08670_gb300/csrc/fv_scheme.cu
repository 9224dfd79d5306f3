// fv_scheme.cu — plain finite-volume stages with a choice of numerical flux
// (Section 2.3.3: HLL, Lax-Friedrichs, Rusanov, Roe, HLLE, HLLC) and of time
// integrator (Heun / SSP-RK2, Eq. 2.19, or SSP-RK3, Eq. 2.20).
//
// The MUSCL-minmod reconstruction (Eq. 2.18), the face-frame rotation (Eq.
// 2.24), the divergence (Eq. 2.23) and the CFL reduction (Eq. 2.10) are those
// of the HLL / SSP-RK2 stage kernels.  Grids with nx a multiple of 4 (>= 8)
// run the row-march kernel of fv_stage.cu with the flux chosen at run time
// (unless the tile variant is asked for); the others this shared-memory tile
// kernel (one uniform branch per face), with four stage kinds:
//   K_FIRST:   q1 = q^n + dt L(q^n)                          (both integrators)
//   K_HEUN:    q^{n+1} = q^n/2 + (q1 + dt L(q1))/2, CFL     (SSP-RK2 stage 2)
//   K_RK3_2:   q2 = 3/4 q^n + 1/4 (q1 + dt L(q1))           (SSP-RK3 stage 2)
//   K_RK3_3:   q^{n+1} = 1/3 q^n + 2/3 (q2 + dt L(q2)), CFL (SSP-RK3 stage 3)
// It also carries the two variants of the shallow-water step that leave the
// periodic flat-bed path (Eq. 2.3, Section 4.2): reflecting walls (the tile's
// halo cells mirror the interior, with the momentum normal to the wall
// negated) and the bed-slope source -g h (dz/dx, dz/dy) with centred slopes of
// the bed z given at the cell centres (mirrored at walls, no sign change).
#include <cuda_runtime.h>

#include "fv_common.cuh"
#include "fv_kernels.h"
#include "fv_schemes.cuh"

namespace fvk {

namespace {

constexpr int TX = 64, TY = 16, SX = TX + 4, SY = TY + 4, NT = 256;
constexpr int ZX = TX + 2, ZY = TY + 2;   // bed tile with a 1-cell halo

template <int C>
constexpr int scheme_smem_bytes() {
  return (C * (SY * SX + TY * (TX + 1) + (TY + 1) * TX) + 4 * (NT / 32) + ZY * ZX) * 4;
}

struct SchemeArgs {
  const float* qin;
  const float* qn;
  float* qout;
  Ctrl* ctrl;
  const DtParams* dp;
  int nx, ny, flux;
  long long plane, member;
  float rdx, rdy, phys;
  int bc;              // BC_PERIODIC or BC_WALL on all four sides
  const float* z;      // bed [ny][nx] (shallow water), or null: flat
};

// Halo index along one axis of length n: periodic wrap, or the mirror image
// (cell -1 - i outside the low end, 2 n - 1 - i outside the high end);
// `flip` is set when the mirror was taken.  A ragged tile also loads cells
// past the two ghost layers the stencil reads; for walls those are clamped
// to the second ghost first, so the mirror stays inside [0, n) for n >= 2.
__device__ __forceinline__ int halo_index(int i, int n, int bc, bool& flip) {
  flip = false;
  if (i >= 0 && i < n) return i;
  if (bc == BC_PERIODIC) return wrap(i, n);
  flip = true;
  i = max(-2, min(i, n + 1));
  return i < 0 ? -1 - i : 2 * n - 1 - i;
}

// Face flux from the four-cell stencil m, a, b, p: MUSCL-minmod face states,
// rotation into the face frame for y faces, the chosen flux, rotation back.
template <int C, int EQ>
__device__ __forceinline__ void face_flux_any(const float (&m)[C], const float (&a)[C], const float (&b)[C],
                                              const float (&p)[C], bool rot, int flux, float phys, float nu,
                                              float (&F)[C]) {
  float L[C], R[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    L[c] = face_left(a[c], minmod(vsub(a[c], m[c]), vsub(b[c], a[c])));
    R[c] = face_right(b[c], minmod(vsub(b[c], a[c]), vsub(p[c], b[c])));
  }
  if (rot) {
    float t = L[1]; L[1] = L[2]; L[2] = t;
    t = R[1]; R[1] = R[2]; R[2] = t;
  }
  if (flux == FLUX_HLL) {
    if constexpr (EQ == SWE) {
      hll_swe<float>(L[0], L[1], L[2], R[0], R[1], R[2], phys, F[0], F[1], F[2]);
    } else {
      hll_euler<float>(L, R, phys, F);
    }
  } else {
    scheme_flux<C, EQ, float>(flux, L, R, phys, nu, F);
  }
  if (rot) {
    float t = F[1]; F[1] = F[2]; F[2] = t;
  }
}

enum { K_FIRST = 0, K_HEUN = 1, K_RK3_2 = 2, K_RK3_3 = 3 };

template <int C, int EQ, int K>
__global__ void __launch_bounds__(NT) stage_scheme_kernel(SchemeArgs a) {
  extern __shared__ float smem[];
  float* sq = smem;                          // [C][SY][SX]
  float* sF = sq + C * SY * SX;              // [C][TY][TX+1]
  float* sG = sF + C * TY * (TX + 1);        // [C][TY+1][TX]
  unsigned* red = reinterpret_cast<unsigned*>(sG + C * (TY + 1) * TX);
  float* zs = reinterpret_cast<float*>(red + 4 * (NT / 32));   // [ZY][ZX]
  constexpr bool last = K == K_HEUN || K == K_RK3_3;

  const int b = blockIdx.z;
  Ctrl* ctrl = a.ctrl + b;
  if (skip_if_done(ctrl)) return;
  const float dt = (float)ctrl->dt;
  // Lax-Friedrichs viscosity per direction: d / (4 dt)
  const float nux = vrcp(vmul(4.f, vmul(dt, a.rdx)));
  const float nuy = vrcp(vmul(4.f, vmul(dt, a.rdy)));
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const float* qin = a.qin + b * a.member;
  const int tid = threadIdx.x;

  for (int idx = tid; idx < C * SY * SX; idx += NT) {
    const int c = idx / (SY * SX);
    const int r = idx - c * (SY * SX);
    const int sy = r / SX, sx = r - sy * SX;
    bool fx, fy;
    const int gx = halo_index(x0 - 2 + sx, a.nx, a.bc, fx), gy = halo_index(y0 - 2 + sy, a.ny, a.bc, fy);
    const float v = qin[c * a.plane + (long long)gy * a.nx + gx];
    // a wall reverses the momentum normal to it (component 1 = x, 2 = y)
    sq[idx] = (c == 1 && fx) || (c == 2 && fy) ? -v : v;
  }
  if (a.z) {
    for (int idx = tid; idx < ZY * ZX; idx += NT) {
      const int sy = idx / ZX, sx = idx - sy * ZX;
      bool fx, fy;
      const int gx = halo_index(x0 - 1 + sx, a.nx, a.bc, fx), gy = halo_index(y0 - 1 + sy, a.ny, a.bc, fy);
      zs[idx] = a.z[(long long)gy * a.nx + gx];
    }
  }
  __syncthreads();

  for (int idx = tid; idx < TY * (TX + 1); idx += NT) {
    const int r = idx / (TX + 1), k = idx - r * (TX + 1);
    const float* row = sq + (r + 2) * SX + k;
    float m[C], s0[C], s1[C], p[C], F[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float* rc = row + c * SY * SX;
      m[c] = rc[0]; s0[c] = rc[1]; s1[c] = rc[2]; p[c] = rc[3];
    }
    face_flux_any<C, EQ>(m, s0, s1, p, false, a.flux, a.phys, nux, F);
#pragma unroll
    for (int c = 0; c < C; ++c) sF[(c * TY + r) * (TX + 1) + k] = F[c];
  }
  for (int idx = tid; idx < (TY + 1) * TX; idx += NT) {
    const int k = idx / TX, i = idx - k * TX;
    const float* col = sq + k * SX + (i + 2);
    float m[C], s0[C], s1[C], p[C], F[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float* cc = col + c * SY * SX;
      m[c] = cc[0]; s0[c] = cc[SX]; s1[c] = cc[2 * SX]; p[c] = cc[3 * SX];
    }
    face_flux_any<C, EQ>(m, s0, s1, p, true, a.flux, a.phys, nuy, F);
#pragma unroll
    for (int c = 0; c < C; ++c) sG[(c * (TY + 1) + k) * TX + i] = F[c];
  }
  __syncthreads();

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
    // bed slope source: -g h (z_e - z_w) / (2 dx), -g h (z_n - z_s) / (2 dy)
    float src1 = 0.f, src2 = 0.f;
    if constexpr (EQ == SWE) {
      if (a.z) {
        const float gh = vmul(a.phys, sq[(r + 2) * SX + i + 2]);
        const float* zc = zs + (r + 1) * ZX + i + 1;
        src1 = vmul(gh, vmul(vsub(zc[1], zc[-1]), 0.5f * a.rdx));
        src2 = vmul(gh, vmul(vsub(zc[ZX], zc[-ZX]), 0.5f * a.rdy));
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float L = divergence<float>(sF[(c * TY + r) * (TX + 1) + i], sF[(c * TY + r) * (TX + 1) + i + 1],
                                  sG[(c * (TY + 1) + r) * TX + i], sG[(c * (TY + 1) + r + 1) * TX + i],
                                  a.rdx, a.rdy);
      if (EQ == SWE && c == 1) L = vsub(L, src1);
      if (EQ == SWE && c == 2) L = vsub(L, src2);
      const float q = sq[(c * SY + r + 2) * SX + i + 2];
      if (K == K_FIRST) {
        out[c] = rk_stage1<float>(q, dt, L);
      } else if (K == K_HEUN) {
        out[c] = rk_stage2<float>(qn[c * a.plane + off], q, 0.5f * dt, L);
      } else {
        // w q^n + (1 - w) (q + dt L), written as q^n + (1 - w) (q + dt L - q^n)
        // so that a constant state stays bitwise constant
        const float qnc = qn[c * a.plane + off];
        out[c] = vfma(K == K_RK3_2 ? 0.25f : 2.f / 3.f, vsub(vfma(dt, L, q), qnc), qnc);
      }
      qout[c * a.plane + off] = out[c];
    }
    if (last) {
      float s;
      if constexpr (EQ == SWE) {
        s = cell_rate_swe(out[0], out[1], out[2], a.phys, a.rdx, a.rdy, bad);
      } else {
        s = cell_rate_euler(out, a.phys, a.rdx, a.rdy, bad);
      }
      amax = fmaxf(amax, s);
    }
  }
  if (last) {
    block_reduce_max_or(amax, bad, red);
    if (tid == 0) publish_and_close(ctrl, a.dp, amax, bad, gridDim.x * gridDim.y, true);
  }
}

template <int C, int EQ, int K>
cudaError_t launch_kind(const SchemeArgs& a, const Geom& g, cudaStream_t s) {
  constexpr int smem = scheme_smem_bytes<C>();
  auto kern = stage_scheme_kernel<C, EQ, K>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, g.B);
  kern<<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int C, int EQ>
cudaError_t launch_eq(int kind, const SchemeArgs& a, const Geom& g, cudaStream_t s) {
  switch (kind) {
    case K_FIRST: return launch_kind<C, EQ, K_FIRST>(a, g, s);
    case K_HEUN: return launch_kind<C, EQ, K_HEUN>(a, g, s);
    case K_RK3_2: return launch_kind<C, EQ, K_RK3_2>(a, g, s);
    default: return launch_kind<C, EQ, K_RK3_3>(a, g, s);
  }
}

cudaError_t launch_scheme_stage(const Geom& g, int kind, int flux, const float* qin, const float* qn,
                                float* qout, Ctrl* ctrl, const DtParams* dp, cudaStream_t s, int bc,
                                const float* z) {
  SchemeArgs a{qin, qn, qout, ctrl, dp, g.nx, g.ny, flux, g.plane(), g.member(),
               (float)(1.0 / g.dx), (float)(1.0 / g.dy), g.phys, bc, z};
  return g.eq == SWE ? launch_eq<3, SWE>(kind, a, g, s) : launch_eq<4, EULER>(kind, a, g, s);
}

}  // namespace

// One step of the plain scheme with the chosen flux and integrator.  q^n is
// qa (updated in place); qb and (SSP-RK3) qc hold the intermediate stages.
cudaError_t enqueue_scheme_step(const Geom& g, int flux, int rk, float* qa, float* qb, float* qc,
                                Ctrl* ctrl, const DtParams* dp, cudaStream_t s, int variant, int bc,
                                const float* z) {
  if (variant != STAGE_TILE && march_supported(g)) {
    // row-march kernels (fv_stage.cu), stage kinds 1..4
    cudaError_t e = launch_stage_general(g, 1, flux, qa, nullptr, qb, ctrl, dp, s, bc, z);
    if (e != cudaSuccess) return e;
    if (rk == 2) return launch_stage_general(g, 2, flux, qb, qa, qa, ctrl, dp, s, bc, z);
    e = launch_stage_general(g, 3, flux, qb, qa, qc, ctrl, dp, s, bc, z);
    if (e != cudaSuccess) return e;
    return launch_stage_general(g, 4, flux, qc, qa, qa, ctrl, dp, s, bc, z);
  }
  cudaError_t e = launch_scheme_stage(g, K_FIRST, flux, qa, nullptr, qb, ctrl, dp, s, bc, z);
  if (e != cudaSuccess) return e;
  if (rk == 2) return launch_scheme_stage(g, K_HEUN, flux, qb, qa, qa, ctrl, dp, s, bc, z);
  e = launch_scheme_stage(g, K_RK3_2, flux, qb, qa, qc, ctrl, dp, s, bc, z);
  if (e != cudaSuccess) return e;
  return launch_scheme_stage(g, K_RK3_3, flux, qc, qa, qa, ctrl, dp, s, bc, z);
}

}  // namespace fvk
