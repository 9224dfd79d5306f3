// fv_sphere.cu — shallow water on the sphere (Sections 2.4 and 4.3).
//
// State q = (h, hu, hv, hw) with a Cartesian momentum m in R^3 on the unit
// sphere, on the logically rectangular two-hemisphere grid: the
// computational rectangle [-3, 1] x [-1, 1] with nx = 2 ny cells, whose
// right square is the upper hemisphere (the disk mapping of Section 2.4 with
// D(d) = d / sqrt 2, R(d) = 1, lifted by z = sqrt(1 - x^2 - y^2), Eq. 2.25)
// and whose left square is the lower one (the disk point of (-2 - xc, yc)).
// x is periodic; above the top row (below the bottom row) lie the same rows
// of the mirrored columns nx - 1 - i.
//
// Per stage (SSP-RK2, Eq. 2.19): MUSCL-minmod face states in the logical
// directions (Eq. 2.18) on the Cartesian variables, rotation to the edge
// frame (n, t, r) (Eq. 2.24 with n, t in R^3), the HLL flux of the 1D problem
// with the t and r momenta passive, rotation back, the flux difference times
// the great-circle edge lengths over the spherical cell area, Eq. 3.1's
// correction F(q_i) . sum_e l_e n_e on the momenta, the Coriolis term of
// Eq. 3.2, and the projection of the momentum onto the tangent plane at the
// cell centre.  The grid metrics are computed once per state in FP64 and
// stored in FP32; every member of a batch shares them.  The other fluxes of
// the planar path (Rusanov, Roe, HLLE, HLLC) treat m.t and m.r as two passive
// variables: the shallow-water solver runs on (h, m.n, m.t) and on
// (h, m.n, m.r), and the second call contributes the flux of m.r.
#include <cuda_runtime.h>

#include "fv_common.cuh"
#include "fv_kernels.h"
#include "fv_schemes.cuh"

namespace fvk {

namespace {

// Metric planes (FP32): x faces [10][ny][nx] (face i between cells i - 1 and
// i: n, t, r, length), y faces [10][ny + 1][nx] (face j between rows j - 1 and
// j), cells [9][ny][nx] (1 / area, centre, sum_e l_e n_e outward, perimeter /
// (2 area), area).
enum { XF_N = 0, XF_T = 3, XF_R = 6, XF_L = 9, F_PLANES = 10 };
enum { C_RA = 0, C_X = 1, C_S = 4, C_RATE = 7, C_AREA = 8, C_PLANES = 9 };

struct SphereLayout {
  long long xf, yf, cell;   // offsets of the three blocks
};

__host__ __device__ inline SphereLayout sphere_layout(int nx, int ny) {
  SphereLayout L;
  L.xf = 0;
  L.yf = (long long)F_PLANES * ny * nx;
  L.cell = L.yf + (long long)F_PLANES * (ny + 1) * nx;
  return L;
}

struct V3 {
  double x, y, z;
};
__device__ inline V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ inline V3 scale(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ inline V3 unit(V3 a) { return scale(a, 1.0 / sqrt(dot(a, a))); }

// Corner (k, j), k = 0..nx, j = 0..ny, on the unit sphere.  A hemisphere's
// square is sampled at s_k = (2 k - ny) / ny so that glued corners are
// computed from identical inputs.  The depth below the disk is written as
// 1 - xp^2 - yp^2 = -b (b + 2 s), b = (d^2 - 1) / (D + sqrt(1 - D^2)), which
// is the same quantity without the cancellation at the rim.
__device__ V3 corner(int k, int j, int ny) {
  const bool upper = k >= ny;
  const int kk = upper ? k - ny : k;
  double xc = (2.0 * kk - ny) / ny;
  const double yc = (2.0 * j - ny) / ny;
  if (!upper) xc = -xc;
  const double d = fmax(fabs(xc), fabs(yc));
  const double D = d * 0.70710678118654752440;
  const double b = (d * d - 1.0) / (D + sqrt(1.0 - D * D));
  const double sd = d > 0.0 ? d : 1.0;
  double xp, yp, s;
  if (fabs(yc) <= fabs(xc)) {
    yp = yc * D / sd;
    s = sqrt(1.0 - yp * yp);
    xp = copysign(1.0, xc) * (b + s);
    if (xc == 0.0) xp = 0.0;
  } else {
    xp = xc * D / sd;
    s = sqrt(1.0 - xp * xp);
    yp = copysign(1.0, yc) * (b + s);
  }
  const double z = sqrt(fmax(-b * (b + 2.0 * s), 0.0));
  return {xp, yp, upper ? z : -z};
}

__device__ V3 cell_centre(int i, int j, int ny) {
  return unit(add(add(corner(i, j, ny), corner(i + 1, j, ny)), add(corner(i, j + 1, ny), corner(i + 1, j + 1, ny))));
}

// Spherical excess of a triangle on the unit sphere.
__device__ double tri_area(V3 a, V3 b, V3 c) {
  return 2.0 * atan2(fabs(dot(a, cross(b, c))), 1.0 + dot(a, b) + dot(b, c) + dot(c, a));
}

// Edge a -> b: length, and the frame t (chord), r (radial through the
// chord's midpoint), n = t x r flipped to point along `dir`.
__device__ void edge_frame(V3 a, V3 b, V3 dir, float* out, long long stride, long long at) {
  const V3 ab = sub(b, a);
  const double chord = sqrt(dot(ab, ab));
  const V3 t = scale(ab, 1.0 / chord);
  const V3 r = unit(add(a, b));
  V3 n = cross(t, r);
  if (dot(n, dir) < 0.0) n = scale(n, -1.0);
  const double v[10] = {n.x, n.y, n.z, t.x, t.y, t.z, r.x, r.y, r.z, 2.0 * asin(fmin(chord * 0.5, 1.0))};
  for (int k = 0; k < 10; ++k) out[k * stride + at] = (float)v[k];
}

// One thread per (face row, column): x face (i, j) for j < ny, y face (i, j)
// for j <= ny.
__global__ void sphere_faces_kernel(float* M, int nx, int ny) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)(ny + 1) * nx) return;
  const int j = (int)(t / nx), i = (int)(t - (long long)j * nx);
  const SphereLayout L = sphere_layout(nx, ny);
  if (j < ny) {
    const V3 dir = sub(cell_centre(i, j, ny), cell_centre(wrap(i - 1, nx), j, ny));
    edge_frame(corner(i, j, ny), corner(i, j + 1, ny), dir, M + L.xf, (long long)ny * nx, (long long)j * nx + i);
  }
  // the cells below and above the y face; across a glued edge the mirrored column
  const V3 below = j > 0 ? cell_centre(i, j - 1, ny) : cell_centre(nx - 1 - i, 0, ny);
  const V3 above = j < ny ? cell_centre(i, j, ny) : cell_centre(nx - 1 - i, ny - 1, ny);
  edge_frame(corner(i, j, ny), corner(i + 1, j, ny), sub(above, below), M + L.yf, (long long)(ny + 1) * nx,
             (long long)j * nx + i);
}

// Cells: 1 / area, centre, sum of l_e n_e over the four edges (outward, from
// the stored FP32 face metrics, as the flux difference sees them), and
// perimeter / (2 area) for the Courant rate.
__global__ void sphere_cells_kernel(float* M, int nx, int ny) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)ny * nx) return;
  const int j = (int)(t / nx), i = (int)(t - (long long)j * nx);
  const SphereLayout L = sphere_layout(nx, ny);
  const long long px = (long long)ny * nx, py = (long long)(ny + 1) * nx;
  const V3 p00 = corner(i, j, ny), p10 = corner(i + 1, j, ny), p01 = corner(i, j + 1, ny), p11 = corner(i + 1, j + 1, ny);
  const double area = tri_area(p00, p10, p11) + tri_area(p00, p11, p01);
  const V3 c = unit(add(add(p00, p10), add(p01, p11)));
  const float* xf = M + L.xf;
  const float* yf = M + L.yf;
  const long long w = (long long)j * nx + i, e = (long long)j * nx + wrap(i + 1, nx);
  const long long s = (long long)j * nx + i, nn = (long long)(j + 1) * nx + i;
  double S[3], per = 0.0;
  for (int k = 0; k < 3; ++k)
    S[k] = (double)xf[XF_L * px + e] * xf[(XF_N + k) * px + e] - (double)xf[XF_L * px + w] * xf[(XF_N + k) * px + w] +
           (double)yf[XF_L * py + nn] * yf[(XF_N + k) * py + nn] - (double)yf[XF_L * py + s] * yf[(XF_N + k) * py + s];
  per = (double)xf[XF_L * px + e] + xf[XF_L * px + w] + yf[XF_L * py + nn] + yf[XF_L * py + s];
  float* cm = M + L.cell;
  const double v[C_PLANES] = {1.0 / area, c.x, c.y, c.z, S[0], S[1], S[2], per / (2.0 * area), area};
  for (int k = 0; k < C_PLANES; ++k) cm[k * px + t] = (float)v[k];
}

// ---------------------------------------------------------------------------
// Stage kernel
// ---------------------------------------------------------------------------
constexpr int TX = 32, TY = 8, SX = TX + 4, SY = TY + 4, NT = 256, C = 4;

struct SphArgs {
  const float* qin;
  const float* qn;
  float* qout;
  const float* M;
  Ctrl* ctrl;
  const DtParams* dp;
  int nx, ny;
  long long plane, member;
  float g, omega;
  int stage;           // 1: q1 = q + dt L(q); 2: Heun's second stage and the CFL reduction
  int B;               // members (looped over inside each block)
  int flux;            // fvk::Flux (HLL, Rusanov, Roe, HLLE or HLLC)
};

__device__ __forceinline__ float mm(float a, float b) {
  return (a * b > 0.f) ? (fabsf(a) < fabsf(b) ? a : b) : 0.f;
}

// HLL flux (Eq. 2.15) in the edge frame: states (h, m_n, m_t, m_r), normal
// flux (m_n, m_n u_n + g h^2 / 2, m_t u_n, m_r u_n).
__device__ void hll4(const float (&L)[C], const float (&R)[C], float g, float (&F)[C]) {
  const float uL = L[1] / L[0], uR = R[1] / R[0];
  const float cL = sqrtf(g * L[0]), cR = sqrtf(g * R[0]);
  const float sL = fminf(uL - cL, uR - cR), sR = fmaxf(uL + cL, uR + cR);
  const float FL[C] = {L[1], L[1] * uL + 0.5f * g * L[0] * L[0], L[2] * uL, L[3] * uL};
  const float FR[C] = {R[1], R[1] * uR + 0.5f * g * R[0] * R[0], R[2] * uR, R[3] * uR};
  if (sL >= 0.f) {
#pragma unroll
    for (int c = 0; c < C; ++c) F[c] = FL[c];
  } else if (sR < 0.f) {
#pragma unroll
    for (int c = 0; c < C; ++c) F[c] = FR[c];
  } else {
    const float inv = 1.f / (sR - sL);
#pragma unroll
    for (int c = 0; c < C; ++c) F[c] = (sR * FL[c] - sL * FR[c] + sL * sR * (R[c] - L[c])) * inv;
  }
}

// Face flux times length from the 4-cell stencil m, a | b, p (Cartesian
// variables) and the face metrics at f (plane stride ps).
__device__ void face_flux(const float (&m)[C], const float (&a)[C], const float (&b)[C], const float (&p)[C],
                          const float* fm, long long ps, long long f, float g, int flux, float (&out)[C]) {
  float Lq[C], Rq[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    Lq[c] = a[c] + 0.5f * mm(a[c] - m[c], b[c] - a[c]);
    Rq[c] = b[c] - 0.5f * mm(b[c] - a[c], p[c] - b[c]);
  }
  float fr[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) fr[k] = fm[k * ps + f];
  const float len = fm[XF_L * ps + f];
  float l[C], r[C], F[C];
  l[0] = Lq[0];
  r[0] = Rq[0];
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    l[1 + v] = Lq[1] * fr[3 * v] + Lq[2] * fr[3 * v + 1] + Lq[3] * fr[3 * v + 2];
    r[1 + v] = Rq[1] * fr[3 * v] + Rq[2] * fr[3 * v + 1] + Rq[3] * fr[3 * v + 2];
  }
  if (flux == FLUX_HLL) {
    hll4(l, r, g, F);
  } else {
    const float lt[3] = {l[0], l[1], l[2]}, rt[3] = {r[0], r[1], r[2]};
    const float lr[3] = {l[0], l[1], l[3]}, rr[3] = {r[0], r[1], r[3]};
    float Ft[3], Fr[3];
    scheme_flux<3, SWE, float>(flux, lt, rt, g, 0.f, Ft);
    scheme_flux<3, SWE, float>(flux, lr, rr, g, 0.f, Fr);
    F[0] = Ft[0];
    F[1] = Ft[1];
    F[2] = Ft[2];
    F[3] = Fr[2];
  }
  out[0] = F[0] * len;
#pragma unroll
  for (int k = 0; k < 3; ++k) out[1 + k] = (F[1] * fr[k] + F[2] * fr[3 + k] + F[3] * fr[6 + k]) * len;
}

// Metric cache of one tile (CACHED instances, dynamic shared memory):
// x faces [10][TY][TX + 1], y faces [10][TY + 1][TX], cells [8][TY][TX].
constexpr int MXP = TY * (TX + 1), MYP = (TY + 1) * TX, MCP = TY * TX;
constexpr int cache_bytes() { return (F_PLANES * MXP + F_PLANES * MYP + C_AREA * MCP) * 4; }

// CACHED: one block per tile looping over the members, with the tile's
// metrics staged in shared memory once for all of them (batches); else one
// block per (tile, member) reading the metrics where they lie (one member).
template <bool CACHED>
__global__ void __launch_bounds__(NT, 4) sphere_stage_kernel(SphArgs a) {
  __shared__ float sq[C][SY][SX];
  __shared__ float sF[C][TY][TX + 1];
  __shared__ float sG[C][TY + 1][TX];
  __shared__ unsigned red[2 * NT / 32];
  extern __shared__ float mcache[];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny;
  const SphereLayout Lm = sphere_layout(nx, ny);
  const long long px = (long long)ny * nx, py = (long long)(ny + 1) * nx;
  // metric planes and strides as the face and cell loops index them
  const float* xm = CACHED ? mcache : a.M + Lm.xf;
  const float* ym = CACHED ? mcache + F_PLANES * MXP : a.M + Lm.yf;
  const float* cmm = CACHED ? mcache + F_PLANES * (MXP + MYP) : a.M + Lm.cell;
  const long long xps = CACHED ? MXP : px, yps = CACHED ? MYP : py, cps = CACHED ? MCP : px;
  if (CACHED) {
    float* cx = mcache;
    float* cy = mcache + F_PLANES * MXP;
    float* cc = mcache + F_PLANES * (MXP + MYP);
    for (int idx = tid; idx < F_PLANES * MXP; idx += NT) {
      const int k = idx / MXP, rr = idx - k * MXP;
      const int r = rr / (TX + 1), c = rr - r * (TX + 1);
      if (y0 + r < ny && x0 + c <= nx) cx[idx] = a.M[Lm.xf + k * px + (long long)(y0 + r) * nx + wrap(x0 + c, nx)];
    }
    for (int idx = tid; idx < F_PLANES * MYP; idx += NT) {
      const int k = idx / MYP, rr = idx - k * MYP;
      const int r = rr / TX, c = rr - r * TX;
      if (y0 + r <= ny && x0 + c < nx) cy[idx] = a.M[Lm.yf + k * py + (long long)(y0 + r) * nx + x0 + c];
    }
    for (int idx = tid; idx < C_AREA * MCP; idx += NT) {
      const int k = idx / MCP, rr = idx - k * MCP;
      const int r = rr / TX, c = rr - r * TX;
      if (y0 + r < ny && x0 + c < nx) cc[idx] = a.M[Lm.cell + k * px + (long long)(y0 + r) * nx + x0 + c];
    }
  }
  const int b0 = CACHED ? 0 : blockIdx.z, b1 = CACHED ? a.B : blockIdx.z + 1;
#pragma unroll 1
  for (int b = b0; b < b1; ++b) {
    Ctrl* ctrl = a.ctrl + b;
    __syncthreads();   // metrics staged / the previous member's tile and fluxes consumed
    if (skip_if_done(ctrl)) continue;
    const float dt = (float)ctrl->dt;
    const float* qin = a.qin + b * a.member;
    // tile with a 2-cell halo: x periodic; beyond the top / bottom row the
    // rows of the mirrored column (rows past the second ghost only occur in
    // a partial tile and are clamped to it)
    for (int idx = tid; idx < C * SY * SX; idx += NT) {
      const int c = idx / (SY * SX), rr = idx - c * SY * SX;
      const int sy = rr / SX, sx = rr - sy * SX;
      int gx = wrap(x0 - 2 + sx, nx);
      int gy = max(-2, min(y0 - 2 + sy, ny + 1));
      if (gy < 0 || gy >= ny) {
        gy = gy < 0 ? -1 - gy : 2 * ny - 1 - gy;
        gx = nx - 1 - gx;
      }
      sq[c][sy][sx] = qin[c * a.plane + (long long)gy * nx + gx];
    }
    __syncthreads();
    for (int idx = tid; idx < TY * (TX + 1); idx += NT) {
      const int r = idx / (TX + 1), k = idx - r * (TX + 1);
      if (y0 + r >= ny || x0 + k > nx) continue;
      float m[C], s0[C], s1[C], p[C], F[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        m[c] = sq[c][r + 2][k];
        s0[c] = sq[c][r + 2][k + 1];
        s1[c] = sq[c][r + 2][k + 2];
        p[c] = sq[c][r + 2][k + 3];
      }
      const long long fx = CACHED ? (long long)r * (TX + 1) + k : (long long)(y0 + r) * nx + wrap(x0 + k, nx);
      face_flux(m, s0, s1, p, xm, xps, fx, a.g, a.flux, F);
#pragma unroll
      for (int c = 0; c < C; ++c) sF[c][r][k] = F[c];
    }
    for (int idx = tid; idx < (TY + 1) * TX; idx += NT) {
      const int k = idx / TX, i = idx - k * TX;
      if (x0 + i >= nx || y0 + k > ny) continue;
      float m[C], s0[C], s1[C], p[C], F[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        m[c] = sq[c][k][i + 2];
        s0[c] = sq[c][k + 1][i + 2];
        s1[c] = sq[c][k + 2][i + 2];
        p[c] = sq[c][k + 3][i + 2];
      }
      const long long fy = CACHED ? (long long)k * TX + i : (long long)(y0 + k) * nx + x0 + i;
      face_flux(m, s0, s1, p, ym, yps, fy, a.g, a.flux, F);
#pragma unroll
      for (int c = 0; c < C; ++c) sG[c][k][i] = F[c];
    }
    __syncthreads();

    float amax = 0.f;
    unsigned bad = 0u;
    const float* qn = a.qn + b * a.member;
    float* qout = a.qout + b * a.member;
    for (int idx = tid; idx < TY * TX; idx += NT) {
      const int r = idx / TX, i = idx - r * TX;
      const int gx = x0 + i, gy = y0 + r;
      if (gx >= nx || gy >= ny) continue;
      const long long off = (long long)gy * nx + gx;
      float q[C];
#pragma unroll
      for (int c = 0; c < C; ++c) q[c] = sq[c][r + 2][i + 2];
      const long long ci = CACHED ? (long long)r * TX + i : off;
      const float ra = cmm[C_RA * cps + ci];
      const float xh[3] = {cmm[C_X * cps + ci], cmm[(C_X + 1) * cps + ci], cmm[(C_X + 2) * cps + ci]};
      const float S[3] = {cmm[C_S * cps + ci], cmm[(C_S + 1) * cps + ci], cmm[(C_S + 2) * cps + ci]};
      // Eq. 3.1's correction on the momenta: F(q) . S = m (m . S) / h + (g h^2 / 2) S
      const float mS = q[1] * S[0] + q[2] * S[1] + q[3] * S[2];
      const float ph = 0.5f * a.g * q[0] * q[0];
      float L[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float net = (sF[c][r][i + 1] - sF[c][r][i]) + (sG[c][r + 1][i] - sG[c][r][i]);
        const float corr = c == 0 ? 0.f : q[c] * (mS / q[0]) + ph * S[c - 1];
        L[c] = -(net - corr) * ra;
      }
      // Coriolis (Eq. 3.2): -2 Omega z (x cross m)
      const float f = -2.f * a.omega * xh[2];
      L[1] += f * (xh[1] * q[3] - xh[2] * q[2]);
      L[2] += f * (xh[2] * q[1] - xh[0] * q[3]);
      L[3] += f * (xh[0] * q[2] - xh[1] * q[1]);
      float out[C];
#pragma unroll
      for (int c = 0; c < C; ++c)
        out[c] = a.stage == 1 ? q[c] + dt * L[c] : 0.5f * qn[c * a.plane + off] + 0.5f * (q[c] + dt * L[c]);
      // project the momentum onto the tangent plane at the cell centre
      const float mx = out[1] * xh[0] + out[2] * xh[1] + out[3] * xh[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) out[1 + k] -= mx * xh[k];
#pragma unroll
      for (int c = 0; c < C; ++c) qout[c * a.plane + off] = out[c];
      if (a.stage == 2) {
        const float h = out[0];
        const float sp = sqrtf(out[1] * out[1] + out[2] * out[2] + out[3] * out[3]) / h + sqrtf(a.g * h);
        const float rate = sp * cmm[C_RATE * cps + ci];
        bad |= (h > 0.f) ? 0u : (unsigned)FV_HEALTH_NONPOSITIVE;
        bad |= (rate < INFINITY) ? 0u : (unsigned)FV_HEALTH_NONFINITE;
        amax = fmaxf(amax, rate);
      }
    }
    if (a.stage == 2) {
      block_reduce_max_or(amax, bad, red);
      if (tid == 0) publish_and_close(ctrl, a.dp, amax, bad, gridDim.x * gridDim.y, true);
    }
  }
}

// Courant rate of a state without advancing time (state creation).
__global__ void sphere_wavespeed_kernel(const float* q, const float* M, Ctrl* ctrl, const DtParams* dp, int nx,
                                        int ny, long long member, float g) {
  __shared__ unsigned red[16];
  const int b = blockIdx.y;
  const long long plane = (long long)nx * ny;
  const float* qb = q + b * member;
  const float* rate_geom = M + sphere_layout(nx, ny).cell + C_RATE * plane;
  float amax = 0.f;
  unsigned bad = 0u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane; i += (long long)gridDim.x * blockDim.x) {
    const float h = qb[i];
    const float m1 = qb[plane + i], m2 = qb[2 * plane + i], m3 = qb[3 * plane + i];
    const float rate = (sqrtf(m1 * m1 + m2 * m2 + m3 * m3) / h + sqrtf(g * h)) * rate_geom[i];
    bad |= (h > 0.f) ? 0u : (unsigned)FV_HEALTH_NONPOSITIVE;
    bad |= (rate < INFINITY) ? 0u : (unsigned)FV_HEALTH_NONFINITE;
    amax = fmaxf(amax, rate);
  }
  block_reduce_max_or(amax, bad, red);
  if (threadIdx.x == 0) publish_and_close(ctrl + b, dp, amax, bad, gridDim.x, false);
}

}  // namespace

long long sphere_metric_floats(int nx, int ny) {
  return sphere_layout(nx, ny).cell + (long long)C_PLANES * ny * nx;
}

// Offsets of the cell centre planes (3) and of the area plane.
long long sphere_centre_offset(int nx, int ny) { return sphere_layout(nx, ny).cell + (long long)C_X * ny * nx; }
long long sphere_area_offset(int nx, int ny) { return sphere_layout(nx, ny).cell + (long long)C_AREA * ny * nx; }

cudaError_t launch_sphere_metrics(float* M, int nx, int ny, cudaStream_t s) {
  const long long nf = (long long)(ny + 1) * nx, nc = (long long)ny * nx;
  sphere_faces_kernel<<<(unsigned)((nf + 127) / 128), 128, 0, s>>>(M, nx, ny);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sphere_cells_kernel<<<(unsigned)((nc + 127) / 128), 128, 0, s>>>(M, nx, ny);
  return cudaGetLastError();
}

cudaError_t launch_sphere_wavespeed(const Geom& g, const float* q, const float* M, Ctrl* ctrl,
                                    const DtParams* dp, cudaStream_t s) {
  long long blocks = (g.plane() + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  dim3 grid((unsigned)blocks, g.B);
  sphere_wavespeed_kernel<<<grid, 256, 0, s>>>(q, M, ctrl, dp, g.nx, g.ny, g.member(), g.phys);
  return cudaGetLastError();
}

cudaError_t enqueue_sphere_step(const Geom& g, int flux, float* qa, float* qb, const float* M, float omega,
                                Ctrl* ctrl, const DtParams* dp, cudaStream_t s) {
  SphArgs a{qa, nullptr, qb, M, ctrl, dp, g.nx, g.ny, g.plane(), g.member(), g.phys, omega, 1, g.B, flux};
  SphArgs b2{qb, qa, qa, M, ctrl, dp, g.nx, g.ny, g.plane(), g.member(), g.phys, omega, 2, g.B, flux};
  // batches share one metric load per tile; a single member reads them directly
  const bool cached = g.B >= 4;
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, cached ? 1 : g.B);
  for (const SphArgs* k : {&a, &b2}) {
    if (cached) {
      sphere_stage_kernel<true><<<grid, NT, cache_bytes(), s>>>(*k);
    } else {
      sphere_stage_kernel<false><<<grid, NT, 0, s>>>(*k);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fvk
