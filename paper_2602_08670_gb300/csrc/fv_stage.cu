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
#include "fv_schemes.cuh"

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
  int flux;            // fvk::Flux of the generic row-march stages
  int bc;              // BC_PERIODIC / BC_WALL (generic row-march stages)
  const float* z;      // shallow-water bed [ny][nx] or null (generic row-march stages)
  int wx0, wx1, wy0, wy1;   // interior [wx0, wx1) x [wy0, wy1): the CFL reduction's cells
};

// The interior window of a geometry (the whole grid unless it carries a ring).
inline void set_window(StageArgs& a, const Geom& g) {
  a.wx0 = g.hx;
  a.wx1 = g.nx - g.hx;
  a.wy0 = g.hy;
  a.wy1 = g.ny - g.hy;
}

// Normal-frame flux of one face from its four-cell stencil.  `rot` selects the
// y-face frame (normal momentum = component 2).
template <int C, int EQ>
__device__ __forceinline__ void stencil_flux(const float (&m)[C], const float (&a)[C],
                                             const float (&b)[C], const float (&p)[C], bool rot,
                                             float phys, float (&F)[C]) {
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
  if constexpr (EQ == SWE) {
    hll_swe<float>(L[0], L[1], L[2], R[0], R[1], R[2], phys, F[0], F[1], F[2]);
  } else {
    hll_euler<float>(L, R, phys, F);
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
      const float L = divergence<float>(Fw, Fe, Gs, Gn, a.rdx, a.rdy);
      const float q = sq[(c * SY + r + 2) * SX + i + 2];
      if (STAGE == 1) {
        out[c] = rk_stage1<float>(q, dt, L);
      } else {
        out[c] = rk_stage2<float>(qn[c * a.plane + off], q, 0.5f * dt, L);
      }
      qout[c * a.plane + off] = out[c];
    }
    if (STAGE == 2) {
      float s;
      unsigned bk = 0u;
      if constexpr (EQ == SWE) {
        s = cell_rate_swe(out[0], out[1], out[2], a.phys, a.rdx, a.rdy, bk);
      } else {
        s = cell_rate_euler(out, a.phys, a.rdx, a.rdy, bk);
      }
      const bool in = gx >= a.wx0 && gx < a.wx1 && gy >= a.wy0 && gy < a.wy1;
      amax = in ? fmaxf(amax, s) : amax;
      bad |= in ? bk : 0u;
    }
  }
  if (STAGE == 2) {
    block_reduce_max_or(amax, bad, red);
    if (tid == 0) publish_and_close(ctrl, a.dp, amax, bad, gridDim.x * gridDim.y, true);
  }
}

// ---------------------------------------------------------------------------
// Row-march stage kernel (nx a multiple of 4).
//
// A block owns a strip of MW = 512 columns (4 per thread, float4 loads) and
// TY rows.  It walks down its rows; the rows it needs (its own plus a 2-row
// periodic halo above and below) arrive through a ring of MS shared-memory
// rows filled by cp.async MPF rows ahead, each with a 2-cell halo on both
// sides.  Per row step a thread
//   - computes the y slopes of its 4 cells at the previous row, the y faces
//     between the two previous rows (rotated HLL) and keeps the lower face
//     state and the last y flux in registers (sliding window down the strip);
//   - computes the x slopes, x faces and x flux divergence of the row being
//     finished from the ring row (its 4 cells plus 2 neighbours each side);
//   - combines and stores that row (float4 stores).
// One __syncthreads per row publishes the ring row.  The y faces are computed
// once; each thread recomputes the x face shared with its right neighbour
// (5 x faces for 4 cells), which removes any per-row flux exchange.
//
// BND instances add reflecting walls and the bed-slope source (Eq. 2.3).
// A wall's ghost cells are the mirror image of the first two interior cells
// with the normal momentum negated: ghost rows are fetched from the mirrored
// rows and their component 2 negated where the y stencil reads them; the
// strip's outer halo pair is fetched in memory order and swapped (component
// 1 negated) where the x stencil reads it.  The bed enters as
// -g h (z_e - z_w) / (2 dx), -g h (z_n - z_s) / (2 dy) on the momenta, with
// the bed mirrored (walls) or wrapped (periodic) across the boundary.
// ---------------------------------------------------------------------------
constexpr int MT = 128;           // threads per block
constexpr int MW = 4 * MT;        // strip width
constexpr int RS = MW + 8;        // ring row stride: 4 left pad (2 used) + MW + 4 right
constexpr int MS = 8;             // ring rows
constexpr int MPF = 3;            // rows prefetched ahead (MS >= MPF + 4: rows r-3 .. r+MPF in use)
static_assert(MS >= MPF + 4, "ring too shallow for the prefetch depth");

template <int C>
constexpr int march_smem_bytes() { return MS * C * RS * 4; }

__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Face flux in the x frame / in the rotated y frame (normal momentum =
// component 2), for scalars or packed pairs.  GEN: the flux is chosen at run
// time (`flux`, fvk::Flux; `nu` the Lax-Friedrichs viscosity of the face's
// direction), packed like the HLL path.
template <int C, int EQ, class V, bool GEN>
__device__ __forceinline__ void normal_flux_any(const V (&L)[C], const V (&R)[C], float phys, int flux,
                                                float nu, V (&F)[C]) {
  if (!GEN || flux == FLUX_HLL) {
    if constexpr (EQ == SWE) {
      hll_swe<V>(L[0], L[1], L[2], R[0], R[1], R[2], phys, F[0], F[1], F[2]);
    } else {
      hll_euler<V>(L, R, phys, F);
    }
  } else {
    scheme_flux<C, EQ, V>(flux, L, R, phys, nu, F);
  }
}

template <int C, int EQ, class V, bool GEN = false>
__device__ __forceinline__ void face_flux_x(const V (&L)[C], const V (&R)[C], float phys, V (&F)[C],
                                            int flux = 0, float nu = 0.f) {
  normal_flux_any<C, EQ, V, GEN>(L, R, phys, flux, nu, F);
}

template <int C, int EQ, class V, bool GEN = false>
__device__ __forceinline__ void face_flux_y(const V (&L)[C], const V (&R)[C], float phys, V (&F)[C],
                                            int flux = 0, float nu = 0.f) {
  V l[C], r[C], f[C];
#pragma unroll
  for (int c = 0; c < C; ++c) { l[c] = L[c]; r[c] = R[c]; }
  l[1] = L[2]; l[2] = L[1];
  r[1] = R[2]; r[2] = R[1];
  normal_flux_any<C, EQ, V, GEN>(l, r, phys, flux, nu, f);
#pragma unroll
  for (int c = 0; c < C; ++c) F[c] = f[c];
  F[1] = f[2]; F[2] = f[1];
}

__device__ __forceinline__ float2 lo(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi(float4 v) { return make_float2(v.z, v.w); }

// STAGE: 1 = q1 = q^n + dt L(q^n); 2 = Heun's second stage (Eq. 2.19) and
// the CFL reduction; with GEN also 3 = SSP-RK3's second stage and 4 = its
// third stage and the CFL reduction (Eq. 2.20).
template <int C, int EQ, int STAGE, bool GEN = false, bool BND = false>
__global__ void __launch_bounds__(MT) stage_march_kernel(StageArgs a, int TY) {
  constexpr bool CFL_STAGE = STAGE == 2 || STAGE == 4;
  extern __shared__ __align__(16) float ring[];   // [MS][C][RS]
  __shared__ unsigned red[2 * MT / 32];
  const int b = blockIdx.z;
  Ctrl* ctrl = a.ctrl + b;
  if (skip_if_done(ctrl)) return;
  const float dt = (float)ctrl->dt;
  // Lax-Friedrichs viscosity per direction (generic stages): d / (4 dt)
  const float nux = GEN ? vrcp(vmul(4.f, vmul(dt, a.rdx))) : 0.f;
  const float nuy = GEN ? vrcp(vmul(4.f, vmul(dt, a.rdy))) : 0.f;
  const int t = threadIdx.x;
  const int X0 = blockIdx.x * MW;
  const int wact = min(MW, a.nx - X0);        // active columns of the strip (multiple of 4)
  const bool active = 4 * t < wact;
  const int Y0 = blockIdx.y * TY;
  const int rows = min(TY, a.ny - Y0);
  const int NL = rows + 4;                    // rows Y0-2 .. Y0+rows+1
  const float* qin = a.qin + b * a.member;
  const bool wall = BND && a.bc == BC_WALL;
  const bool wall_w = wall && X0 == 0;                  // the strip touches the west wall
  const bool wall_e = wall && X0 + wact == a.nx;        // ... the east wall
  // left / right halo cells xl, xl+1 and xr, xr+1 (at a wall: the two
  // boundary cells in memory order, mirrored when read)
  const int xl = X0 == 0 ? (wall ? 0 : a.nx - 2) : X0 - 2;
  const int xr = X0 + wact == a.nx ? (wall ? a.nx - 2 : 0) : X0 + wact;
  const int plane = (int)a.plane;                       // < 2^31 floats per variable plane
  int gy_next = Y0 - 2;                                 // next row to fetch (periodic)
  while (gy_next < 0) gy_next += a.ny;
  int i_next = 0;

  auto issue_next = [&]() {
    float* slot = ring + ((unsigned)i_next % MS) * C * RS;
    int gy = gy_next;
    if (wall) {
      // virtual row Y0 - 2 + i_next lies in [-2, ny + 1]: mirror it inside
      const int v = Y0 - 2 + i_next;
      gy = v < 0 ? -1 - v : (v >= a.ny ? 2 * a.ny - 1 - v : v);
    }
    const float* src = qin + gy * a.nx;
    if (active) {
#pragma unroll
      for (int c = 0; c < C; ++c) cp_async16(slot + c * RS + 4 + 4 * t, src + c * plane + X0 + 4 * t);
    }
    if (t == 0) {
#pragma unroll
      for (int c = 0; c < C; ++c) cp_async8(slot + c * RS + 2, src + c * plane + xl);
    } else if (t == 1) {
#pragma unroll
      for (int c = 0; c < C; ++c) cp_async8(slot + c * RS + 4 + wact, src + c * plane + xr);
    }
    ++i_next;
    if (++gy_next == a.ny) gy_next = 0;
  };

#pragma unroll
  for (int p = 0; p < MPF; ++p) {
    if (p < NL) issue_next();
    cp_async_commit();
  }

  float2 PL[C][2];   // lower state of the next y face (row r-1 extrapolated up), cell pairs
  float2 Gp[C][2];   // y flux on the south face of the row being finished
  float amax = 0.f;
  unsigned bad = 0u;
  const float* qnb = a.qn + b * a.member;
  float* qout = a.qout + b * a.member;
  const int col = 4 + 4 * t;

  for (int i = 0; i < NL; ++i) {
    if (i + MPF < NL) issue_next();
    cp_async_commit();
    const int orow = Y0 + i - 4;                // output row at this step (valid for i >= 4)
    float2 qn2[C][2];
    if (STAGE >= 2 && i >= 4 && active) {
      const int off = orow * a.nx + X0 + 4 * t;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(qnb + c * plane + off));
        qn2[c][0] = lo(v);
        qn2[c][1] = hi(v);
      }
    }
    // bed around the 4 cells of the output row: zr[0..5] = columns
    // 4t-1 .. 4t+4 of the row, zs / zn the rows below / above
    float zr[6], zs[4], zn[4];
    if constexpr (BND && EQ == SWE) {
      if (a.z && i >= 4 && active) {
        const int x = X0 + 4 * t;
        const int xw = x > 0 ? x - 1 : (wall ? 0 : a.nx - 1);
        const int xe = x + 4 < a.nx ? x + 4 : (wall ? a.nx - 1 : 0);
        const int ys = orow > 0 ? orow - 1 : (wall ? 0 : a.ny - 1);
        const int yn = orow + 1 < a.ny ? orow + 1 : (wall ? a.ny - 1 : 0);
        const float4 c4 = __ldg(reinterpret_cast<const float4*>(a.z + orow * a.nx + x));
        const float4 s4 = __ldg(reinterpret_cast<const float4*>(a.z + ys * a.nx + x));
        const float4 n4 = __ldg(reinterpret_cast<const float4*>(a.z + yn * a.nx + x));
        zr[0] = __ldg(a.z + orow * a.nx + xw);
        zr[1] = c4.x; zr[2] = c4.y; zr[3] = c4.z; zr[4] = c4.w;
        zr[5] = __ldg(a.z + orow * a.nx + xe);
        zs[0] = s4.x; zs[1] = s4.y; zs[2] = s4.z; zs[3] = s4.w;
        zn[0] = n4.x; zn[1] = n4.y; zn[2] = n4.z; zn[3] = n4.w;
      }
    }
    cp_async_wait<MPF>();
    __syncthreads();
    if (i < 2 || !active) continue;

    const float* s0 = ring + ((unsigned)(i - 2) % MS) * C * RS;   // row r-2
    const float* s1 = ring + ((unsigned)(i - 1) % MS) * C * RS;   // row r-1
    const float* s2 = ring + ((unsigned)i % MS) * C * RS;         // row r
    // a ghost row behind a wall carries the mirrored normal momentum -hv
    float m0 = 1.f, m1 = 1.f, m2 = 1.f;
    if (wall) {
      const int v0r = Y0 + i - 4, v1r = v0r + 1, v2r = v0r + 2;   // virtual rows of s0, s1, s2
      m0 = v0r < 0 || v0r >= a.ny ? -1.f : 1.f;
      m1 = v1r < 0 || v1r >= a.ny ? -1.f : 1.f;
      m2 = v2r < 0 || v2r >= a.ny ? -1.f : 1.f;
    }
    float2 q0[C][2], q1[C][2], sy[C][2];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float4 v0 = *reinterpret_cast<const float4*>(s0 + c * RS + col);
      float4 v1 = *reinterpret_cast<const float4*>(s1 + c * RS + col);
      float4 v2 = *reinterpret_cast<const float4*>(s2 + c * RS + col);
      if (BND && c == 2) {
        v0 = make_float4(m0 * v0.x, m0 * v0.y, m0 * v0.z, m0 * v0.w);
        v1 = make_float4(m1 * v1.x, m1 * v1.y, m1 * v1.z, m1 * v1.w);
        v2 = make_float4(m2 * v2.x, m2 * v2.y, m2 * v2.z, m2 * v2.w);
      }
      q0[c][0] = lo(v0); q0[c][1] = hi(v0);
      q1[c][0] = lo(v1); q1[c][1] = hi(v1);
      // y slope at row r-1
      sy[c][0] = minmod(vsub(q1[c][0], q0[c][0]), vsub(lo(v2), q1[c][0]));
      sy[c][1] = minmod(vsub(q1[c][1], q0[c][1]), vsub(hi(v2), q1[c][1]));
    }

    if (i >= 3) {
      // y faces between rows r-2 and r-1 (two packed cell pairs)
      float2 Gn[C][2];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float2 Lf[C], Rf[C], F[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          Lf[c] = PL[c][p];
          Rf[c] = face_right(q1[c][p], sy[c][p]);
        }
        face_flux_y<C, EQ, float2, GEN>(Lf, Rf, a.phys, F, a.flux, nuy);
#pragma unroll
        for (int c = 0; c < C; ++c) Gn[c][p] = F[c];
      }
      if (i >= 4) {
        // finish row r-2: cells 4t-2 .. 4t+5 of the ring row, slopes at
        // 4t-1 .. 4t+4, faces 4t-1/2 .. 4t+7/2 (pairs f0 f1, f2 f3; f4 alone)
        float e[C][8];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float2 lft = *reinterpret_cast<const float2*>(s0 + c * RS + col - 2);
          const float2 rgt = *reinterpret_cast<const float2*>(s0 + c * RS + col + 4);
          e[c][0] = lft.x; e[c][1] = lft.y;
          e[c][2] = q0[c][0].x; e[c][3] = q0[c][0].y; e[c][4] = q0[c][1].x; e[c][5] = q0[c][1].y;
          e[c][6] = rgt.x; e[c][7] = rgt.y;
          if (BND) {
            // wall ghosts: cell -2 = cell 1, -1 = cell 0 (and nx, nx+1 = nx-1,
            // nx-2), normal momentum negated
            const float sg = c == 1 ? -1.f : 1.f;
            if (wall_w && t == 0) {
              e[c][0] = sg * lft.y;
              e[c][1] = sg * lft.x;
            }
            if (wall_e && 4 * t + 4 == wact) {
              e[c][6] = sg * rgt.y;
              e[c][7] = sg * rgt.x;
            }
          }
        }
        float sx[C][6];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          float d[7];
#pragma unroll
          for (int j = 0; j < 7; ++j) d[j] = vsub(e[c][j + 1], e[c][j]);
#pragma unroll
          for (int j = 0; j < 6; ++j) sx[c][j] = minmod(d[j], d[j + 1]);
        }
        float2 Fx2[C][2];
        float Fx4[C];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          float2 Lf[C], Rf[C], F[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            Lf[c] = face_left(make_float2(e[c][1 + 2 * p], e[c][2 + 2 * p]),
                              make_float2(sx[c][2 * p], sx[c][2 * p + 1]));
            Rf[c] = face_right(make_float2(e[c][2 + 2 * p], e[c][3 + 2 * p]),
                               make_float2(sx[c][2 * p + 1], sx[c][2 * p + 2]));
          }
          face_flux_x<C, EQ, float2, GEN>(Lf, Rf, a.phys, F, a.flux, nux);
#pragma unroll
          for (int c = 0; c < C; ++c) Fx2[c][p] = F[c];
        }
        {
          float Lf[C], Rf[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            Lf[c] = face_left(e[c][5], sx[c][4]);
            Rf[c] = face_right(e[c][6], sx[c][5]);
          }
          face_flux_x<C, EQ, float, GEN>(Lf, Rf, a.phys, Fx4, a.flux, nux);
        }
        // faces f0..f4 = Fx2[.][0].x, Fx2[.][0].y, Fx2[.][1].x, Fx2[.][1].y, Fx4
        float2 out[C][2];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float2 Fw0 = Fx2[c][0];
          const float2 Fe0 = make_float2(Fx2[c][0].y, Fx2[c][1].x);
          const float2 Fw1 = Fx2[c][1];
          const float2 Fe1 = make_float2(Fx2[c][1].y, Fx4[c]);
          float2 L0 = divergence(Fw0, Fe0, Gp[c][0], Gn[c][0], a.rdx, a.rdy);
          float2 L1 = divergence(Fw1, Fe1, Gp[c][1], Gn[c][1], a.rdx, a.rdy);
          if constexpr (BND && EQ == SWE) {
            if (a.z && c > 0) {
              // bed slope: -g h (z_e - z_w) / (2 dx) on hu, -g h (z_n - z_s) / (2 dy) on hv
              float sk[4];
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float h = (k & 1) ? q0[0][k >> 1].y : q0[0][k >> 1].x;
                const float gh = vmul(a.phys, h);
                sk[k] = c == 1 ? vmul(gh, vmul(vsub(zr[k + 2], zr[k]), 0.5f * a.rdx))
                               : vmul(gh, vmul(vsub(zn[k], zs[k]), 0.5f * a.rdy));
              }
              L0 = vsub(L0, make_float2(sk[0], sk[1]));
              L1 = vsub(L1, make_float2(sk[2], sk[3]));
            }
          }
          if (STAGE == 1) {
            out[c][0] = rk_stage1(q0[c][0], dt, L0);
            out[c][1] = rk_stage1(q0[c][1], dt, L1);
          } else if (STAGE == 2) {
            out[c][0] = rk_stage2(qn2[c][0], q0[c][0], 0.5f * dt, L0);
            out[c][1] = rk_stage2(qn2[c][1], q0[c][1], 0.5f * dt, L1);
          } else {
            // SSP-RK3: q^n + (1 - w)(q + dt L - q^n), 1 - w = 1/4 or 2/3
            const float2 w = vsplat<float2>(STAGE == 3 ? 0.25f : 2.f / 3.f);
            const float2 d = vsplat<float2>(dt);
            out[c][0] = vfma(w, vsub(vfma(d, L0, q0[c][0]), qn2[c][0]), qn2[c][0]);
            out[c][1] = vfma(w, vsub(vfma(d, L1, q0[c][1]), qn2[c][1]), qn2[c][1]);
          }
        }
        const int off = orow * a.nx + X0 + 4 * t;
#pragma unroll
        for (int c = 0; c < C; ++c)
          *reinterpret_cast<float4*>(qout + c * plane + off) =
              make_float4(out[c][0].x, out[c][0].y, out[c][1].x, out[c][1].y);
        if (CFL_STAGE) {
          const bool row_in = orow >= a.wy0 && orow < a.wy1;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            float v[C];
#pragma unroll
            for (int c = 0; c < C; ++c) v[c] = (k & 1) ? out[c][k >> 1].y : out[c][k >> 1].x;
            float sp;
            unsigned bk = 0u;
            if constexpr (EQ == SWE) {
              sp = cell_rate_swe(v[0], v[1], v[2], a.phys, a.rdx, a.rdy, bk);
            } else {
              sp = cell_rate_euler(v, a.phys, a.rdx, a.rdy, bk);
            }
            const int x = X0 + 4 * t + k;
            const bool in = row_in && x >= a.wx0 && x < a.wx1;
            amax = in ? fmaxf(amax, sp) : amax;
            bad |= in ? bk : 0u;
          }
        }
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        Gp[c][0] = Gn[c][0];
        Gp[c][1] = Gn[c][1];
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      PL[c][0] = face_left(q1[c][0], sy[c][0]);
      PL[c][1] = face_left(q1[c][1], sy[c][1]);
    }
  }
  cp_async_wait<0>();
  if (CFL_STAGE) {
    block_reduce_max_or(amax, bad, red);
    if (t == 0) publish_and_close(ctrl, a.dp, amax, bad, gridDim.x * gridDim.y, true);
  }
}

template <int C, int EQ>
__global__ void __launch_bounds__(256) wavespeed_init_kernel(const float* q, Ctrl* ctrl,
                                                             const DtParams* dp, int nx, int ny,
                                                             long long plane, long long member,
                                                             float phys, float rdx, float rdy, int hx,
                                                             int hy, int b0) {
  __shared__ unsigned red[16];
  const int b = b0 + blockIdx.y;
  const float* qb = q + b * member;
  float amax = 0.f;
  unsigned bad = 0u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / nx), x = (int)(i - (long long)y * nx);
    if (x < hx || x >= nx - hx || y < hy || y >= ny - hy) continue;   // ring of a subdomain
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
                                                               double phys, int nx, int ny, int hx,
                                                               int hy) {
  __shared__ double sh[DIAG_NT];
  const int b = blockIdx.y;
  const float* qb = q + b * member;
  double acc[C + 1];
#pragma unroll
  for (int c = 0; c <= C; ++c) acc[c] = 0.0;
  for (long long i = blockIdx.x * (long long)DIAG_NT + threadIdx.x; i < plane;
       i += (long long)DIAG_BLOCKS * DIAG_NT) {
    if (hx | hy) {
      const int y = (int)(i / nx), x = (int)(i - (long long)y * nx);
      if (x < hx || x >= nx - hx || y < hy || y >= ny - hy) continue;   // ring of a subdomain
    }
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
  c->done = c->exhausted | (c->step_end > 0 && c->step >= c->step_end ? 1u : 0u);
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

// Rows per march block: long strips amortise the 4 halo rows, but the grid
// must fill the GPU in whole waves.  Among TY in [8, 128] pick the one whose
// last wave is fullest (ties: larger TY).
int march_rows_per_block(int ny, int columns_x_members, int per_sm) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
  }
  const long long slots = (long long)sms * per_sm;
  int best = ny < 8 ? ny : 8;
  double best_eff = -1.0;
  for (int ty = 8; ty <= 128; ++ty) {
    if (ty > ny && ty != 8) break;
    const long long blocks = (long long)columns_x_members * ((ny + ty - 1) / ty);
    const long long waves = (blocks + slots - 1) / slots;
    // useful fraction: block work over wave slots, discounting the halo rows
    const double eff = (double)blocks / (double)(waves * slots) * (double)ty / (ty + 4.0);
    if (eff >= best_eff) {
      best_eff = eff;
      best = ty;
    }
  }
  return best;
}

template <int C, int EQ, int STAGE, bool GEN, bool BND = false>
cudaError_t launch_march(const StageArgs& a, const Geom& g, cudaStream_t s) {
  constexpr int smem = march_smem_bytes<C>();
  auto kern = stage_march_kernel<C, EQ, STAGE, GEN, BND>;
  static int per_sm = 0;   // resident blocks per SM, queried once per instance
  if (!per_sm) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, MT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  const int nsx = (g.nx + MW - 1) / MW;
  const int TY = march_rows_per_block(g.ny, nsx * g.B, per_sm);
  dim3 grid(nsx, (g.ny + TY - 1) / TY, g.B);
  kern<<<grid, MT, smem, s>>>(a, TY);
  return cudaGetLastError();
}

template <int C, int EQ, bool BND>
cudaError_t launch_general_b(const StageArgs& a, const Geom& g, int stage, cudaStream_t s) {
  switch (stage) {
    case 1: return launch_march<C, EQ, 1, true, BND>(a, g, s);
    case 2: return launch_march<C, EQ, 2, true, BND>(a, g, s);
    case 3: return launch_march<C, EQ, 3, true, BND>(a, g, s);
    default: return launch_march<C, EQ, 4, true, BND>(a, g, s);
  }
}

template <int C, int EQ>
cudaError_t launch_general_t(const Geom& g, int stage, int flux, const float* qin, const float* qn,
                             float* qout, Ctrl* ctrl, const DtParams* dp, cudaStream_t s, int bc,
                             const float* z) {
  StageArgs a{qin, qn, qout, ctrl, dp, g.nx, g.ny, g.plane(), g.member(),
              (float)(1.0 / g.dx), (float)(1.0 / g.dy), g.phys, flux, bc, z};
  set_window(a, g);
  if (bc != BC_PERIODIC || z) return launch_general_b<C, EQ, true>(a, g, stage, s);
  return launch_general_b<C, EQ, false>(a, g, stage, s);
}

template <int C, int EQ, int STAGE>
cudaError_t launch_stage_t(const Geom& g, const float* qin, const float* qn, float* qout,
                           Ctrl* ctrl, const DtParams* dp, cudaStream_t s, int variant) {
  StageArgs a{qin, qn, qout, ctrl, dp, g.nx, g.ny, g.plane(), g.member(),
              (float)(1.0 / g.dx), (float)(1.0 / g.dy), g.phys, 0};
  set_window(a, g);
  const bool march_ok = (g.nx % 4 == 0) && g.nx >= 8;
  if (variant == STAGE_MARCH && !march_ok) return cudaErrorInvalidValue;
  if (variant != STAGE_TILE && march_ok) return launch_march<C, EQ, STAGE, false>(a, g, s);
  constexpr int smem = stage_smem_bytes<C>();
  auto kern = stage_minmod_kernel<C, EQ, STAGE>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, g.B);
  kern<<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stage_minmod(const Geom& g, int stage, const float* qin, const float* qn,
                                float* qout, Ctrl* ctrl, const DtParams* dp, cudaStream_t s,
                                int variant) {
  if (g.eq == SWE) {
    return stage == 1 ? launch_stage_t<3, SWE, 1>(g, qin, qn, qout, ctrl, dp, s, variant)
                      : launch_stage_t<3, SWE, 2>(g, qin, qn, qout, ctrl, dp, s, variant);
  }
  return stage == 1 ? launch_stage_t<4, EULER, 1>(g, qin, qn, qout, ctrl, dp, s, variant)
                    : launch_stage_t<4, EULER, 2>(g, qin, qn, qout, ctrl, dp, s, variant);
}

bool march_supported(const Geom& g) { return (g.nx % 4 == 0) && g.nx >= 8; }

cudaError_t launch_stage_general(const Geom& g, int stage, int flux, const float* qin, const float* qn,
                                 float* qout, Ctrl* ctrl, const DtParams* dp, cudaStream_t s, int bc,
                                 const float* z) {
  if (!march_supported(g)) return cudaErrorInvalidValue;
  if ((bc == BC_WALL && g.ny < 2) || (z && g.eq != SWE)) return cudaErrorInvalidValue;
  return g.eq == SWE ? launch_general_t<3, SWE>(g, stage, flux, qin, qn, qout, ctrl, dp, s, bc, z)
                     : launch_general_t<4, EULER>(g, stage, flux, qin, qn, qout, ctrl, dp, s, bc, z);
}

cudaError_t launch_wavespeed_init(const Geom& g, const float* q, Ctrl* ctrl, const DtParams* dp,
                                  cudaStream_t s, int member) {
  long long blocks = (g.plane() + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  const int b0 = member < 0 ? 0 : member;
  dim3 grid((unsigned)blocks, member < 0 ? g.B : 1);
  if (g.eq == SWE) {
    wavespeed_init_kernel<3, SWE><<<grid, 256, 0, s>>>(q, ctrl, dp, g.nx, g.ny, g.plane(),
                                                       g.member(), g.phys, (float)(1.0 / g.dx),
                                                       (float)(1.0 / g.dy), g.hx, g.hy, b0);
  } else {
    wavespeed_init_kernel<4, EULER><<<grid, 256, 0, s>>>(q, ctrl, dp, g.nx, g.ny, g.plane(),
                                                         g.member(), g.phys, (float)(1.0 / g.dx),
                                                         (float)(1.0 / g.dy), g.hx, g.hy, b0);
  }
  return cudaGetLastError();
}

long long diag_partials_size(const Geom& g) { return (long long)g.B * (g.C + 1) * DIAG_BLOCKS; }

cudaError_t launch_diagnostics(const Geom& g, const float* q, double* partials, double* out,
                               cudaStream_t s) {
  dim3 grid(DIAG_BLOCKS, g.B);
  if (g.eq == SWE) {
    diag_partial_kernel<3, SWE><<<grid, DIAG_NT, 0, s>>>(q, partials, g.plane(), g.member(),
                                                         g.phys_d, g.nx, g.ny, g.hx, g.hy);
  } else {
    diag_partial_kernel<4, EULER><<<grid, DIAG_NT, 0, s>>>(q, partials, g.plane(), g.member(),
                                                           g.phys_d, g.nx, g.ny, g.hx, g.hy);
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
