// fv_train.cu — training of the learned-stencil network on the GPU.
//
// A taped forward rollout of T learned SSP-RK2 steps (fixed dt) keeps every
// stage input, the CNN activations and the coefficients; the rollout loss of
// Eq. 2.28 gives the cotangents of the predicted states; the backward walks
// the steps in reverse through
//   stage 2: q' = q/2 + q1/2 + (dt/2) L(q1),   stage 1: q1 = q + dt L(q),
// where the vector-Jacobian product of L is the adjoint of the flux
// divergence, of the HLL flux (Eq. 2.15, on the branch taken) and of the
// reconstruction (learned stencils, or minmod where the positivity fallback
// was taken), plus the CNN backward for the coefficients' dependence on q.
// The face-state network (third approach) has no direct path from q to the
// faces: the adjoint of its stage gives the cotangents of the side states
// (one HLL VJP per face), and the CNN backward turns them into dq.
#include <cuda_runtime.h>

#include <vector>

#include "fv_common.cuh"
#include <cuda_bf16.h>

#include "fv_internal.h"
#include "stencil_net.cuh"

namespace fvk {
namespace {

constexpr int AX = 32, AY = 16, ANT = 256;
constexpr int QX = AX + 6, QY = AY + 6;       // q staged with a 3-cell halo
constexpr int MX = AX + 4, MY = AY + 4;       // cotangent staged with a 2-cell halo
constexpr int FXN = AX + 3, FYN = AY + 3;     // faces touching the tile, per row / column

constexpr int adj_smem_bytes() {
  return (3 * QY * QX + 3 * MY * MX + AY * FXN * 12 + FYN * AX * 12) * 4;
}

struct AdjArgs {
  const float* q;       // stage input [B][3][plane]
  const float* w;       // coefficients [B][36][plane]
  const float* hmin;    // [B]
  const float* lam;     // cotangent of the stage output [B][3][plane]; that of L(q) is mu_scale * lam
  float mu_scale;
  float* gq;            // out: VJP w.r.t. q (reconstruction + flux path) [B][3][plane]
  uint16_t* dr;         // out: VJP w.r.t. the network's raw outputs, BF16 [B][6][plane][8]
  int nx, ny;
  long long plane;
  float rdx, rdy, g;
};

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Cotangent of the 18 coefficients of one face direction of a cell (its 6
// sum-to-one triples) -> cotangent of the raw outputs behind them (Section
// 2.5.3's normalisation w = r - mean(r) + e: subtract each triple's mean),
// BF16, written into the cell's records of dr.  x faces are channels 0..17
// (records 0, 1 and the first word of record 2), y faces 18..35 (the rest of
// record 2, records 3 and 4) plus the zero padding 36..47 (end of record 4,
// record 5).
__device__ __forceinline__ void store_raw_cotangent(uint16_t* dr, long long plane, int b, long long cell,
                                                    bool ydir, const float (&gwd)[18]) {
  float r[18];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const float m = (gwd[3 * t] + gwd[3 * t + 1] + gwd[3 * t + 2]) * (1.f / 3.f);
    r[3 * t] = gwd[3 * t] - m;
    r[3 * t + 1] = gwd[3 * t + 1] - m;
    r[3 * t + 2] = gwd[3 * t + 2] - m;
  }
  auto rec = [&](int g) { return reinterpret_cast<uint32_t*>(dr + (((long long)b * 6 + g) * plane + cell) * 8); };
  if (!ydir) {
    *reinterpret_cast<uint4*>(rec(0)) = make_uint4(pack2(r[0], r[1]), pack2(r[2], r[3]), pack2(r[4], r[5]),
                                                   pack2(r[6], r[7]));
    *reinterpret_cast<uint4*>(rec(1)) = make_uint4(pack2(r[8], r[9]), pack2(r[10], r[11]), pack2(r[12], r[13]),
                                                   pack2(r[14], r[15]));
    rec(2)[0] = pack2(r[16], r[17]);
  } else {
    uint32_t* r2 = rec(2);
    r2[1] = pack2(r[0], r[1]);
    *reinterpret_cast<uint2*>(r2 + 2) = make_uint2(pack2(r[2], r[3]), pack2(r[4], r[5]));
    *reinterpret_cast<uint4*>(rec(3)) = make_uint4(pack2(r[6], r[7]), pack2(r[8], r[9]), pack2(r[10], r[11]),
                                                   pack2(r[12], r[13]));
    *reinterpret_cast<uint4*>(rec(4)) = make_uint4(pack2(r[14], r[15]), pack2(r[16], r[17]), 0u, 0u);
    *reinterpret_cast<uint4*>(rec(5)) = make_uint4(0u, 0u, 0u, 0u);
  }
}

// VJP of the face-frame SWE HLL flux (three-branch form, written with the
// clamped speeds zL = min(sL, 0), zR = max(sR, 0)): given mu = dLoss/dF,
// accumulate dLoss/dL and dLoss/dR.
__device__ void hll_swe_vjp(const float (&L)[3], const float (&R)[3], float g, const float (&mu)[3],
                            float (&dL)[3], float (&dR)[3]) {
  const float hL = L[0], mL = L[1], tL = L[2], hR = R[0], mR = R[1], tR = R[2];
  const float rL = 1.f / hL, rR = 1.f / hR;
  const float uL = mL * rL, uR = mR * rR;
  const float cL = sqrtf(g * hL), cR = sqrtf(g * hR);
  const float a1 = uL - cL, a2 = uR - cR, b1 = uL + cL, b2 = uR + cR;
  const float sL = fminf(a1, a2), sR = fmaxf(b1, b2);
  const float zL = fminf(sL, 0.f), zR = fmaxf(sR, 0.f);
  const float inv = 1.f / (zR - zL);
  const float FL[3] = {mL, mL * uL + 0.5f * g * hL * hL, tL * uL};
  const float FR[3] = {mR, mR * uR + 0.5f * g * hR * hR, tR * uR};
  float gFL[3], gFR[3], gzL = 0.f, gzR = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float d = R[c] - L[c];
    const float F = (zR * FL[c] - zL * FR[c] + zL * zR * d) * inv;
    gFL[c] = mu[c] * zR * inv;
    gFR[c] = -mu[c] * zL * inv;
    const float gd = mu[c] * zL * zR * inv;
    dR[c] += gd;
    dL[c] -= gd;
    gzL += mu[c] * (F - FR[c] + zR * d) * inv;
    gzR += mu[c] * (FL[c] - F + zL * d) * inv;
  }
  const float gsL = sL < 0.f ? gzL : 0.f;
  const float gsR = sR > 0.f ? gzR : 0.f;
  const bool leftmin = a1 <= a2, leftmax = b1 >= b2;
  const float guL = (leftmin ? gsL : 0.f) + (leftmax ? gsR : 0.f);
  const float gcL = (leftmin ? -gsL : 0.f) + (leftmax ? gsR : 0.f);
  const float guR = (leftmin ? 0.f : gsL) + (leftmax ? 0.f : gsR);
  const float gcR = (leftmin ? 0.f : -gsL) + (leftmax ? 0.f : gsR);
  // left side: FL = (m, m u + g h^2 / 2, t u), u = m / h, c = sqrt(g h)
  {
    float du = guL + gFL[1] * mL + gFL[2] * tL;
    dL[0] += gFL[1] * g * hL + gcL * 0.5f * g / cL - du * uL * rL;
    dL[1] += gFL[0] + gFL[1] * uL + du * rL;
    dL[2] += gFL[2] * uL;
  }
  {
    float du = guR + gFR[1] * mR + gFR[2] * tR;
    dR[0] += gFR[1] * g * hR + gcR * 0.5f * g / cR - du * uR * rR;
    dR[1] += gFR[0] + gFR[1] * uR + du * rR;
    dR[2] += gFR[2] * uR;
  }
}

// d minmod(d1, d2) / d(d1, d2) on the branch taken (ab <= 0: 0; |a| < |b|: a; else b).
__device__ __forceinline__ void minmod_grad(float d1, float d2, float& g1, float& g2) {
  if (!(d1 * d2 > 0.f)) {
    g1 = 0.f;
    g2 = 0.f;
  } else if (fabsf(d1) < fabsf(d2)) {
    g1 = 1.f;
    g2 = 0.f;
  } else {
    g1 = 0.f;
    g2 = 1.f;
  }
}

// One face: stencil q[k] = Q_{i-1+k} (k = 0..3, per variable), owner weights
// wd[18], cotangent of the face flux muF (face frame already applied by the
// caller through `rot`).  Adds the cotangents of the 4 stencil cells to
// cq[4][3] and writes the coefficient cotangents to gwd[18] (zero if the
// fallback was taken).
__device__ void face_vjp(const float (&q)[4][3], const float (&wd)[18], float hmin, float g,
                         bool rot, const float (&muF)[3], float (&cq)[4][3], float (&gwd)[18]) {
  float L[3], R[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* wl = wd + (c * 2 + 0) * 3;
    const float* wr = wd + (c * 2 + 1) * 3;
    L[c] = vfma(wl[2], q[2][c], vfma(wl[1], q[1][c], vmul(wl[0], q[0][c])));
    R[c] = vfma(wr[2], q[3][c], vfma(wr[1], q[2][c], vmul(wr[0], q[1][c])));
  }
  const bool fallback = !(L[0] >= hmin) || !(R[0] >= hmin);
  if (fallback) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      L[c] = face_left(q[1][c], minmod(vsub(q[1][c], q[0][c]), vsub(q[2][c], q[1][c])));
      R[c] = face_right(q[2][c], minmod(vsub(q[2][c], q[1][c]), vsub(q[3][c], q[2][c])));
    }
  }
  // face frame: y faces carry (h, hv, hu)
  float l[3] = {L[0], rot ? L[2] : L[1], rot ? L[1] : L[2]};
  float r[3] = {R[0], rot ? R[2] : R[1], rot ? R[1] : R[2]};
  float mu[3] = {muF[0], rot ? muF[2] : muF[1], rot ? muF[1] : muF[2]};
  float dl[3] = {0.f, 0.f, 0.f}, dr[3] = {0.f, 0.f, 0.f};
  hll_swe_vjp(l, r, g, mu, dl, dr);
  const float dLq[3] = {dl[0], rot ? dl[2] : dl[1], rot ? dl[1] : dl[2]};
  const float dRq[3] = {dr[0], rot ? dr[2] : dr[1], rot ? dr[1] : dr[2]};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (fallback) {
      float g1, g2;
      minmod_grad(q[1][c] - q[0][c], q[2][c] - q[1][c], g1, g2);
      // L = q1 + s/2, s = mm(q1 - q0, q2 - q1)
      cq[0][c] += dLq[c] * (-0.5f * g1);
      cq[1][c] += dLq[c] * (1.f + 0.5f * g1 - 0.5f * g2);
      cq[2][c] += dLq[c] * (0.5f * g2);
      minmod_grad(q[2][c] - q[1][c], q[3][c] - q[2][c], g1, g2);
      // R = q2 - t/2, t = mm(q2 - q1, q3 - q2)
      cq[1][c] += dRq[c] * (0.5f * g1);
      cq[2][c] += dRq[c] * (1.f - 0.5f * g1 + 0.5f * g2);
      cq[3][c] += dRq[c] * (-0.5f * g2);
#pragma unroll
      for (int k = 0; k < 6; ++k) gwd[c * 6 + k] = 0.f;
    } else {
      const float* wl = wd + (c * 2 + 0) * 3;
      const float* wr = wd + (c * 2 + 1) * 3;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cq[k][c] += wl[k] * dLq[c];
        cq[k + 1][c] += wr[k] * dRq[c];
        gwd[c * 6 + k] = q[k][c] * dLq[c];
        gwd[c * 6 + 3 + k] = q[k + 1][c] * dRq[c];
      }
    }
  }
}

__global__ void __launch_bounds__(ANT) learned_adjoint_kernel(AdjArgs a) {
  extern __shared__ float sm[];
  float* sq = sm;                          // [3][QY][QX]
  float* smu = sq + 3 * QY * QX;           // [3][MY][MX]
  float* cx = smu + 3 * MY * MX;           // [AY][FXN][4][3]
  float* cy = cx + AY * FXN * 12;          // [FYN][AX][4][3]
  const int b = blockIdx.z;
  const int x0 = blockIdx.x * AX, y0 = blockIdx.y * AY;
  const int tid = threadIdx.x;
  const float* qb = a.q + (long long)b * 3 * a.plane;
  const float* mb = a.lam + (long long)b * 3 * a.plane;
  const float* wb = a.w + (long long)b * 36 * a.plane;
  const float hmin = a.hmin[b];
  for (int i = tid; i < 3 * QY * QX; i += ANT) {
    const int c = i / (QY * QX), r = (i / QX) % QY, s = i % QX;
    sq[i] = qb[c * a.plane + (long long)wrap(y0 - 3 + r, a.ny) * a.nx + wrap(x0 - 3 + s, a.nx)];
  }
  for (int i = tid; i < 3 * MY * MX; i += ANT) {
    const int c = i / (MY * MX), r = (i / MX) % MY, s = i % MX;
    smu[i] = a.mu_scale * mb[c * a.plane + (long long)wrap(y0 - 2 + r, a.ny) * a.nx + wrap(x0 - 2 + s, a.nx)];
  }
  __syncthreads();
  // x faces: owner i = x0 - 2 + f, f = 0..AX+2, on tile rows
  for (int e = tid; e < AY * FXN; e += ANT) {
    const int r = e / FXN, f = e - r * FXN;
    const int gy = y0 + r;
    float q[4][3], wd[18], mu[3], cq[4][3] = {}, gwd[18];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) q[k][c] = sq[(c * QY + r + 3) * QX + f + k];
    const long long owner = (long long)wrap(gy, a.ny) * a.nx + wrap(x0 - 2 + f, a.nx);
#pragma unroll
    for (int j = 0; j < 18; ++j) wd[j] = wb[j * a.plane + owner];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      mu[c] = (smu[(c * MY + r + 2) * MX + f + 1] - smu[(c * MY + r + 2) * MX + f]) * a.rdx;
    face_vjp(q, wd, hmin, a.g, false, mu, cq, gwd);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) cx[(e * 4 + k) * 3 + c] = cq[k][c];
    if (f >= 2 && f < AX + 2 && gy < a.ny && x0 - 2 + f < a.nx)
      store_raw_cotangent(a.dr, a.plane, b, owner, false, gwd);
  }
  // y faces: owner j = y0 - 2 + f on tile columns
  for (int e = tid; e < FYN * AX; e += ANT) {
    const int f = e / AX, i = e - f * AX;
    const int gx = x0 + i;
    float q[4][3], wd[18], mu[3], cq[4][3] = {}, gwd[18];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) q[k][c] = sq[(c * QY + f + k) * QX + i + 3];
    const long long owner = (long long)wrap(y0 - 2 + f, a.ny) * a.nx + wrap(gx, a.nx);
#pragma unroll
    for (int j = 0; j < 18; ++j) wd[j] = wb[(18 + j) * a.plane + owner];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      mu[c] = (smu[(c * MY + f + 1) * MX + i + 2] - smu[(c * MY + f) * MX + i + 2]) * a.rdy;
    face_vjp(q, wd, hmin, a.g, true, mu, cq, gwd);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) cy[(e * 4 + k) * 3 + c] = cq[k][c];
    if (f >= 2 && f < AY + 2 && y0 - 2 + f < a.ny && gx < a.nx)
      store_raw_cotangent(a.dr, a.plane, b, owner, true, gwd);
  }
  __syncthreads();
  // gather: cell (r, i) gets contribution k from the face whose owner is
  // cell - 1 + k, i.e. face index f = i + 3 - k (x) / r + 3 - k (y)
  float* gqb = a.gq + (long long)b * 3 * a.plane;
  for (int e = tid; e < AY * AX; e += ANT) {
    const int r = e / AX, i = e - r * AX;
    const int gx = x0 + i, gy = y0 + r;
    if (gx >= a.nx || gy >= a.ny) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        s += cx[((r * FXN + i + 3 - k) * 4 + k) * 3 + c];
        s += cy[(((r + 3 - k) * AX + i) * 4 + k) * 3 + c];
      }
      gqb[c * a.plane + (long long)gy * a.nx + gx] = s;
    }
  }
}

// Adjoint of one face-state stage: mu = dLoss/dL(q) per cell.  The face
// between cells i-1 and i carries F = HLL(E_{i-1}, W_i) with
// dLoss/dF = (mu_i - mu_{i-1}) / dx; its VJP is the cotangent of exactly those
// two side states (each side state meets one face), written once.  The
// thread of cell i handles its west and south faces.
__global__ void face_adjoint_kernel(const float* sides, const float* mu, float* gs, int nx, int ny,
                                    long long plane, long long cells, float rdx, float rdy, float g) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= cells) return;
  const long long b = t / plane, cell = t - b * plane;
  const int y = (int)(cell / nx), x = (int)(cell - (long long)y * nx);
  const float* sb = sides + b * 12 * plane;
  const float* mb = mu + b * 3 * plane;
  float* gb = gs + b * 12 * plane;
  {
    const long long cl = (long long)y * nx + wrap(x - 1, nx);
    float L[3], R[3], m[3], dl[3] = {0.f, 0.f, 0.f}, dr[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      L[v] = sb[(3 * 1 + v) * plane + cl];      // east side of the west cell
      R[v] = sb[(3 * 0 + v) * plane + cell];    // west side of this cell
      m[v] = (mb[v * plane + cell] - mb[v * plane + cl]) * rdx;
    }
    hll_swe_vjp(L, R, g, m, dl, dr);
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      gb[(3 * 1 + v) * plane + cl] = dl[v];
      gb[(3 * 0 + v) * plane + cell] = dr[v];
    }
  }
  {
    const long long cs = (long long)wrap(y - 1, ny) * nx + x;
    float L[3], R[3], m[3], dl[3] = {0.f, 0.f, 0.f}, dr[3] = {0.f, 0.f, 0.f};
    // face frame of a y face: (h, hv, hu)
    const int perm[3] = {0, 2, 1};
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      L[v] = sb[(3 * 3 + perm[v]) * plane + cs];      // north side of the south cell
      R[v] = sb[(3 * 2 + perm[v]) * plane + cell];    // south side of this cell
      m[v] = (mb[perm[v] * plane + cell] - mb[perm[v] * plane + cs]) * rdy;
    }
    hll_swe_vjp(L, R, g, m, dl, dr);
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      gb[(3 * 3 + perm[v]) * plane + cs] = dl[v];
      gb[(3 * 2 + perm[v]) * plane + cell] = dr[v];
    }
  }
}

// out = alpha * x + beta * y + gamma * z (elementwise, any of y, z may be null).
__global__ void axpbypcz_kernel(float* out, const float* x, float alpha, const float* y, float beta,
                                const float* z, float gamma, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = alpha * x[i];
  if (y) v += beta * y[i];
  if (z) v += gamma * z[i];
  out[i] = v;
}

// Eq. 2.28: loss = sum_t sum_c mean_{b,cells} ((pred - target) / scale_c)^2 and
// its gradient w.r.t. pred; per-block FP64 partial sums.
// Eq. 2.28 over the recorded rollout: blockIdx.x = plane (step t, member b,
// variable c in [T][B][3] order), blockIdx.y = part of the plane; FP32 differences scaled by 1 /
// scale_c, squared and summed per thread, then per block in FP64; the host
// adds the block sums in a fixed order.  grad receives d loss / d q.
__global__ void __launch_bounds__(256) rollout_loss_kernel(const float* pred, const float* target, float* grad,
                                                           double* part, long long plane, double inv_count,
                                                           float is0, float is1, float is2, float gscale) {
  __shared__ double sh[256];
  const int c = (int)(blockIdx.x % 3);
  const float is = c == 0 ? is0 : (c == 1 ? is1 : is2);
  const long long base = (long long)blockIdx.x * plane;
  float acc = 0.f;
  for (long long i = blockIdx.y * (long long)blockDim.x + threadIdx.x; i < plane;
       i += (long long)gridDim.y * blockDim.x) {
    const float d = (pred[base + i] - target[base + i]) * is;
    acc = fmaf(d, d, acc);
    if (grad) grad[base + i] = gscale * d * is;
  }
  sh[threadIdx.x] = (double)acc;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)blockIdx.x * gridDim.y + blockIdx.y] = sh[0] * inv_count;
}

// Adam (bias-corrected) on the FP32 master parameters.
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void fixed_ctrl_kernel(Ctrl* c, int B, double dt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  c[b] = Ctrl{};
  c[b].dt = dt;
}

}  // namespace

cudaError_t launch_learned_adjoint(const Geom& g, const float* q, const float* w, const float* hmin,
                                   const float* lam, float mu_scale, float* gq, uint16_t* dr, cudaStream_t s) {
  constexpr int smem = adj_smem_bytes();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(learned_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  AdjArgs a{q, w, hmin, lam, mu_scale, gq, dr, g.nx, g.ny, g.plane(), (float)(1.0 / g.dx), (float)(1.0 / g.dy), g.phys};
  dim3 grid((g.nx + AX - 1) / AX, (g.ny + AY - 1) / AY, g.B);
  learned_adjoint_kernel<<<grid, ANT, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_axpbypcz(float* out, const float* x, float alpha, const float* y, float beta,
                            const float* z, float gamma, long long n, cudaStream_t s) {
  axpbypcz_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, x, alpha, y, beta, z, gamma, n);
  return cudaGetLastError();
}

cudaError_t launch_face_adjoint(const Geom& g, const float* sides, const float* mu, float* gs, cudaStream_t s) {
  const long long cells = (long long)g.B * g.plane();
  face_adjoint_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(
      sides, mu, gs, g.nx, g.ny, g.plane(), cells, (float)(1.0 / g.dx), (float)(1.0 / g.dy), g.phys);
  return cudaGetLastError();
}

}  // namespace fvk

// ---------------------------------------------------------------------------
// Tape of a learned rollout
// ---------------------------------------------------------------------------
struct fv_tape {
  fv_net* net = nullptr;
  fvk::Geom g{};
  int T = 0;
  double dt = 0.0;
  cudaStream_t stream = nullptr;
  float* states = nullptr;      // q_0 .. q_T  [T+1][B][3][plane]
  float* stage1 = nullptr;      // q1_0 .. q1_{T-1} [T][B][3][plane]
  float* coeffs = nullptr;      // w per stage [2T][B][36][plane] (face-state: side states [2T][B][12][plane])
  bool face = false;            // the network is a face-state network
  snk::Acts* acts = nullptr;    // per stage [2T]
  float* hmin = nullptr;        // [B]
  fvk::Ctrl* ctrl = nullptr;
  fvk::DtParams* dp = nullptr;
  snk::Grads grads;
  float *lam = nullptr, *lam1 = nullptr, *mu = nullptr, *gq = nullptr, *gw = nullptr;
  double* loss_part = nullptr;
  float* dsn = nullptr;         // gradient of the last loss w.r.t. q_1 .. q_T
  double hmin_frac = 1e-3;
  bool have_forward = false;
  // the backward's launch sequence, captured once (after one direct run)
  // and replayed; keyed by the caller's buffers
  cudaGraphExec_t bwd_exec = nullptr;
  const float* bwd_dsn = nullptr;
  const float* bwd_dparams = nullptr;
  const float* bwd_dq0 = nullptr;
  int bwd_calls = 0;
  bool bwd_graph_off = false;   // a capture failed: run directly from then on
  // the forward's launches after the copy of q0, likewise (keyed by snaps)
  cudaGraphExec_t fwd_exec = nullptr;
  const float* fwd_snaps = nullptr;
  int fwd_calls = 0;
  bool fwd_graph_off = false;
};

namespace fvk {
cudaError_t launch_learned_adjoint(const Geom& g, const float* q, const float* w, const float* hmin,
                                   const float* lam, float mu_scale, float* gq, uint16_t* dr, cudaStream_t s);
cudaError_t launch_axpbypcz(float* out, const float* x, float alpha, const float* y, float beta,
                            const float* z, float gamma, long long n, cudaStream_t s);
cudaError_t launch_face_adjoint(const Geom& g, const float* sides, const float* mu, float* gs, cudaStream_t s);
}  // namespace fvk

namespace {

// blocks per plane of the loss kernel (about 2048 cells per block)
inline int loss_blocks_x(long long plane) {
  long long bx = (plane + 2047) / 2048;
  if (bx > 65535) bx = 65535;
  return (int)(bx < 1 ? 1 : bx);
}

// h_min per member = frac * mean depth (FP64 sum of h over the member).
__global__ void hmin_kernel(const float* q, float* hmin, long long plane, double frac) {
  __shared__ double sh[256];
  const int b = blockIdx.x;
  const float* h = q + (long long)b * 3 * plane;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < plane; i += 256) acc += h[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) hmin[b] = (float)(frac * sh[0] / (double)plane);
}

void tape_free(fv_tape* t) {
  if (!t) return;
  if (t->stream) cudaStreamSynchronize(t->stream);
  cudaFree(t->states);
  cudaFree(t->stage1);
  cudaFree(t->coeffs);
  if (t->acts) {
    for (int k = 0; k < 2 * t->T; ++k) snk::acts_free(t->acts[k]);
    delete[] t->acts;
  }
  cudaFree(t->hmin);
  cudaFree(t->ctrl);
  cudaFree(t->dp);
  if (t->bwd_exec) cudaGraphExecDestroy(t->bwd_exec);
  if (t->fwd_exec) cudaGraphExecDestroy(t->fwd_exec);
  snk::backward_free(t->grads);
  cudaFree(t->lam);
  cudaFree(t->lam1);
  cudaFree(t->mu);
  cudaFree(t->gq);
  cudaFree(t->gw);
  cudaFree(t->loss_part);
  cudaFree(t->dsn);
  if (t->stream) cudaStreamDestroy(t->stream);
  delete t;
}

long long st_count(const fv_tape* t) { return (long long)t->g.B * 3 * t->g.plane(); }

}  // namespace

extern "C" int fv_tape_create(fv_net* net, int B, int ny, int nx, int T, double dt, double g,
                              double hmin_frac, fv_tape** out) {
  if (!net || !out) return fvh::fail(FV_EINVAL, "null argument");
  *out = nullptr;
  if (B < 1 || T < 1 || !(dt > 0) || !(g > 0) || hmin_frac < 0 || hmin_frac >= 1)
    return fvh::fail(FV_EINVAL, "bad tape arguments");
  if (!snk::grid_supported(nx) || ((long long)nx * ny) % snk::TILE != 0)
    return fvh::fail(FV_EINVAL, "unsupported grid for the learned step");
  fv_tape* t = new fv_tape();
  t->net = net;
  t->face = net->n.kind == snk::NET_FACE;
  const int nout = t->face ? snk::N_OUT_FACE : snk::N_OUT;
  t->T = T;
  t->dt = dt;
  t->g.nx = nx;
  t->g.ny = ny;
  t->g.B = B;
  t->g.C = 3;
  t->g.eq = fvk::SWE;
  t->g.dx = 1.0 / nx;
  t->g.dy = 1.0 / ny;
  t->g.phys = (float)g;
  t->g.phys_d = g;
  const long long cells = (long long)B * nx * ny, sc = 3 * cells;
  cudaError_t e = cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&t->states, sizeof(float) * sc * (T + 1));
  if (e == cudaSuccess) e = cudaMalloc(&t->stage1, sizeof(float) * sc * T);
  if (e == cudaSuccess) e = cudaMalloc(&t->coeffs, sizeof(float) * nout * cells * 2 * T);
  if (e == cudaSuccess) {
    t->acts = new snk::Acts[2 * T];
    for (int k = 0; k < 2 * T && e == cudaSuccess; ++k) e = snk::acts_reserve(t->acts[k], cells, t->face);
  }
  if (e == cudaSuccess) e = cudaMalloc(&t->hmin, sizeof(float) * B);
  if (e == cudaSuccess) e = cudaMalloc(&t->ctrl, sizeof(fvk::Ctrl) * B);
  if (e == cudaSuccess) e = cudaMalloc(&t->dp, sizeof(fvk::DtParams));
  if (e == cudaSuccess) e = snk::backward_reserve(t->grads, cells, snk::backward_partials_floats(B, ny, nx));
  if (e == cudaSuccess) e = cudaMalloc(&t->lam, sizeof(float) * sc);
  if (e == cudaSuccess) e = cudaMalloc(&t->lam1, sizeof(float) * sc);
  if (e == cudaSuccess) e = cudaMalloc(&t->mu, sizeof(float) * sc);
  if (e == cudaSuccess) e = cudaMalloc(&t->gq, sizeof(float) * sc);
  if (e == cudaSuccess) e = cudaMalloc(&t->gw, sizeof(float) * nout * cells);
  if (e == cudaSuccess)
    e = cudaMalloc(&t->loss_part, sizeof(double) * (size_t)T * B * 3 * loss_blocks_x((long long)nx * ny));
  if (e == cudaSuccess) e = cudaMalloc(&t->dsn, sizeof(float) * sc * T);
  if (e == cudaSuccess) {
    fvk::DtParams dp{};
    dp.mode = FV_DT_FIXED;
    dp.dt_fixed = dt;
    e = cudaMemcpy(t->dp, &dp, sizeof dp, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    tape_free(t);
    return fvh::cuda_fail(e, "fv_tape_create");
  }
  t->hmin_frac = hmin_frac;
  *out = t;
  return FV_OK;
}

extern "C" int fv_tape_destroy(fv_tape* t) {
  tape_free(t);
  return FV_OK;
}

namespace {
// The forward's launches after the copy of q0 into the tape (stream s).
int tape_forward_enqueue(fv_tape* t, float* snaps, cudaStream_t s) {
  const long long sc = st_count(t), plane = t->g.plane();
  hmin_kernel<<<t->g.B, 256, 0, s>>>(t->states, t->hmin, plane, t->hmin_frac);
  FV_CUDA_TRY(cudaGetLastError());
  fvk::fixed_ctrl_kernel<<<(t->g.B + 127) / 128, 128, 0, s>>>(t->ctrl, t->g.B, t->dt);
  FV_CUDA_TRY(cudaGetLastError());
  const snk::Net& N = t->net->n;
  const long long wsz = (t->face ? 4 : 12) * sc;   // 12 or 36 planes per member
  for (int n = 0; n < t->T; ++n) {
    float* qn = t->states + sc * n;
    float* q1 = t->stage1 + sc * n;
    float* w0 = t->coeffs + wsz * (2 * n);
    float* w1 = t->coeffs + wsz * (2 * n + 1);
    if (t->face) {
      FV_CUDA_TRY(snk::forward_faces(N, qn, t->g.B, t->g.ny, t->g.nx, t->acts[2 * n], w0, nullptr, s));
      FV_CUDA_TRY(fvk::launch_stage_face(t->g, 1, qn, nullptr, q1, w0, t->ctrl, t->dp, s));
      FV_CUDA_TRY(snk::forward_faces(N, q1, t->g.B, t->g.ny, t->g.nx, t->acts[2 * n + 1], w1, nullptr, s));
      FV_CUDA_TRY(fvk::launch_stage_face(t->g, 2, q1, qn, qn + sc, w1, t->ctrl, t->dp, s));
      continue;
    }
    FV_CUDA_TRY(snk::forward(N, qn, t->g.B, t->g.ny, t->g.nx, t->acts[2 * n], w0, nullptr, s));
    FV_CUDA_TRY(fvk::launch_stage_learned(t->g, 1, qn, nullptr, q1, w0, t->hmin, t->ctrl, t->dp, s));
    FV_CUDA_TRY(snk::forward(N, q1, t->g.B, t->g.ny, t->g.nx, t->acts[2 * n + 1], w1, nullptr, s));
    FV_CUDA_TRY(fvk::launch_stage_learned(t->g, 2, q1, qn, qn + sc, w1, t->hmin, t->ctrl, t->dp, s));
  }
  if (snaps)
    FV_CUDA_TRY(cudaMemcpyAsync(snaps, t->states + sc, sizeof(float) * sc * t->T,
                                cudaMemcpyDeviceToDevice, s));
  return FV_OK;
}
}  // namespace

// As the backward: the first call runs directly, later calls with the same
// snaps buffer replay a captured graph of the launches after the copy of q0.
extern "C" int fv_tape_forward(fv_tape* t, const float* q0, float* snaps) {
  if (!t || !q0) return fvh::fail(FV_EINVAL, "null argument");
  const long long sc = st_count(t);
  cudaStream_t s = t->stream;
  FV_CUDA_TRY(cudaMemcpyAsync(t->states, q0, sizeof(float) * sc, cudaMemcpyDeviceToDevice, s));
  const bool graph = !t->fwd_graph_off && t->fwd_calls++ > 0;
  if (!graph) {
    const int rc = tape_forward_enqueue(t, snaps, s);
    if (rc != FV_OK) return rc;
  } else {
    if (t->fwd_exec && t->fwd_snaps != snaps) {
      cudaGraphExecDestroy(t->fwd_exec);
      t->fwd_exec = nullptr;
    }
    bool direct = false;
    if (!t->fwd_exec) {
      cudaGraph_t gr = nullptr;
      FV_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const int rc = tape_forward_enqueue(t, snaps, s);
      const cudaError_t ce = cudaStreamEndCapture(s, &gr);
      cudaError_t ie = cudaErrorUnknown;
      if (rc == FV_OK && ce == cudaSuccess) ie = cudaGraphInstantiate(&t->fwd_exec, gr, 0);
      if (gr) cudaGraphDestroy(gr);
      if (rc != FV_OK || ce != cudaSuccess || ie != cudaSuccess) {
        cudaGetLastError();
        t->fwd_exec = nullptr;
        t->fwd_graph_off = true;
        direct = true;
        const int rc2 = tape_forward_enqueue(t, snaps, s);
        if (rc2 != FV_OK) return rc2;
      } else {
        t->fwd_snaps = snaps;
      }
    }
    if (!direct) FV_CUDA_TRY(cudaGraphLaunch(t->fwd_exec, s));
  }
  FV_CUDA_TRY(cudaStreamSynchronize(s));
  t->have_forward = true;
  std::vector<fvk::Ctrl> c(t->g.B);
  FV_CUDA_TRY(cudaMemcpy(c.data(), t->ctrl, sizeof(fvk::Ctrl) * t->g.B, cudaMemcpyDeviceToHost));
  for (int b = 0; b < t->g.B; ++b)
    if (c[b].health) return fvh::fail(FV_EUNSTABLE, "learned rollout became unstable");
  return fvs::net_check(t->net);
}

extern "C" int fv_tape_loss(fv_tape* t, const float* targets, const float* scale3, double* loss) {
  if (!t || !targets || !scale3 || !loss) return fvh::fail(FV_EINVAL, "null argument");
  if (!t->have_forward) return fvh::fail(FV_EINVAL, "fv_tape_forward has not run");
  const long long sc = st_count(t);
  const int bx = loss_blocks_x(t->g.plane());
  const int planes = t->T * t->g.B * 3;
  const double inv_count = 1.0 / (double)((long long)t->g.B * t->g.plane());
  fvk::rollout_loss_kernel<<<dim3(planes, bx), 256, 0, t->stream>>>(
      t->states + sc, targets, t->dsn, t->loss_part, t->g.plane(), inv_count, (float)(1.0 / scale3[0]),
      (float)(1.0 / scale3[1]), (float)(1.0 / scale3[2]), (float)(2.0 * inv_count));
  FV_CUDA_TRY(cudaGetLastError());
  std::vector<double> part((size_t)bx * planes);
  FV_CUDA_TRY(cudaMemcpyAsync(part.data(), t->loss_part, sizeof(double) * part.size(),
                              cudaMemcpyDeviceToHost, t->stream));
  FV_CUDA_TRY(cudaStreamSynchronize(t->stream));
  double sum = 0.0;
  for (double v : part) sum += v;
  *loss = sum;
  return FV_OK;
}

namespace {
// Every launch of the tape's backward on stream s (and the backward's own
// side streams, joined back into s).
int tape_backward_enqueue(fv_tape* t, const float* dsn, float* dparams, float* dq0, cudaStream_t s) {
  const long long sc = st_count(t);
  const snk::Net& N = t->net->n;
  const float dt = (float)t->dt;
  const int B = t->g.B, ny = t->g.ny, nx = t->g.nx;
  FV_CUDA_TRY(cudaMemcpyAsync(t->lam, dsn + sc * (t->T - 1), sizeof(float) * sc,
                              cudaMemcpyDeviceToDevice, s));
  const long long wsz = (t->face ? 4 : 12) * sc;
  for (int n = t->T - 1; n >= 0; --n) {
    const float* qn = t->states + sc * n;
    const float* q1 = t->stage1 + sc * n;
    const float* w0 = t->coeffs + wsz * (2 * n);
    const float* w1 = t->coeffs + wsz * (2 * n + 1);
    if (t->face) {
      // stage 2: q' = q/2 + q1/2 + (dt/2) L(q1), L through the side states only
      FV_CUDA_TRY(fvk::launch_axpbypcz(t->mu, t->lam, 0.5f * dt, nullptr, 0.f, nullptr, 0.f, sc, s));
      FV_CUDA_TRY(fvk::launch_face_adjoint(t->g, w1, t->mu, t->gw, s));
      FV_CUDA_TRY(cudaMemsetAsync(t->gq, 0, sizeof(float) * sc, s));
      FV_CUDA_TRY(snk::backward_faces(N, q1, B, ny, nx, t->acts[2 * n + 1], w1, t->gw, t->gq, dparams, 1.f,
                                      t->grads, s));
      FV_CUDA_TRY(fvk::launch_axpbypcz(t->lam1, t->lam, 0.5f, t->gq, 1.f, nullptr, 0.f, sc, s));
      // stage 1: q1 = q + dt L(q)
      FV_CUDA_TRY(fvk::launch_axpbypcz(t->mu, t->lam1, dt, nullptr, 0.f, nullptr, 0.f, sc, s));
      FV_CUDA_TRY(fvk::launch_face_adjoint(t->g, w0, t->mu, t->gw, s));
      FV_CUDA_TRY(cudaMemsetAsync(t->gq, 0, sizeof(float) * sc, s));
      FV_CUDA_TRY(snk::backward_faces(N, qn, B, ny, nx, t->acts[2 * n], w0, t->gw, t->gq, dparams, 1.f,
                                      t->grads, s));
      FV_CUDA_TRY(fvk::launch_axpbypcz(t->lam, t->lam, 0.5f, t->lam1, 1.f, t->gq, 1.f, sc, s));
      if (n >= 1)
        FV_CUDA_TRY(fvk::launch_axpbypcz(t->lam, t->lam, 1.f, dsn + sc * (n - 1), 1.f, nullptr, 0.f, sc, s));
      continue;
    }
    // stage 2 (the adjoint takes mu = (dt/2) lam and writes the cotangent of
    // the network's raw outputs)
    FV_CUDA_TRY(fvk::launch_learned_adjoint(t->g, q1, w1, t->hmin, t->lam, 0.5f * dt, t->gq, t->grads.dr, s));
    FV_CUDA_TRY(snk::backward_from_raw(N, q1, B, ny, nx, t->acts[2 * n + 1], t->gq, dparams, 1.f, t->grads, s));
    FV_CUDA_TRY(fvk::launch_axpbypcz(t->lam1, t->lam, 0.5f, t->gq, 1.f, nullptr, 0.f, sc, s));
    // stage 1 (mu = dt lam1)
    FV_CUDA_TRY(fvk::launch_learned_adjoint(t->g, qn, w0, t->hmin, t->lam1, dt, t->gq, t->grads.dr, s));
    FV_CUDA_TRY(snk::backward_from_raw(N, qn, B, ny, nx, t->acts[2 * n], t->gq, dparams, 1.f, t->grads, s));
    FV_CUDA_TRY(fvk::launch_axpbypcz(t->lam, t->lam, 0.5f, t->lam1, 1.f, t->gq, 1.f, sc, s));
    if (n >= 1)
      FV_CUDA_TRY(fvk::launch_axpbypcz(t->lam, t->lam, 1.f, dsn + sc * (n - 1), 1.f, nullptr, 0.f, sc, s));
  }
  if (dq0) FV_CUDA_TRY(cudaMemcpyAsync(dq0, t->lam, sizeof(float) * sc, cudaMemcpyDeviceToDevice, s));
  return FV_OK;
}
}  // namespace

// The first call runs the launches directly (one-time set-up such as kernel
// attributes happens there); later calls with the same buffers replay a CUDA
// graph captured from the same sequence, which removes the per-launch host
// and scheduling gaps of its ~300 launches.  The arithmetic is the same.
extern "C" int fv_tape_backward(fv_tape* t, const float* dsnaps, float* dparams, float* dq0) {
  if (!t || !dparams) return fvh::fail(FV_EINVAL, "null argument");
  if (!t->have_forward) return fvh::fail(FV_EINVAL, "fv_tape_forward has not run");
  const float* dsn = dsnaps ? dsnaps : t->dsn;
  cudaStream_t s = t->stream;
  const bool graph = !t->bwd_graph_off && t->bwd_calls++ > 0;
  if (!graph) {
    const int rc = tape_backward_enqueue(t, dsn, dparams, dq0, s);
    if (rc != FV_OK) return rc;
  } else {
    if (t->bwd_exec && (t->bwd_dsn != dsn || t->bwd_dparams != dparams || t->bwd_dq0 != dq0)) {
      cudaGraphExecDestroy(t->bwd_exec);
      t->bwd_exec = nullptr;
    }
    if (!t->bwd_exec) {
      cudaGraph_t gr = nullptr;
      FV_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const int rc = tape_backward_enqueue(t, dsn, dparams, dq0, s);
      const cudaError_t ce = cudaStreamEndCapture(s, &gr);
      cudaError_t ie = cudaErrorUnknown;
      if (rc == FV_OK && ce == cudaSuccess) ie = cudaGraphInstantiate(&t->bwd_exec, gr, 0);
      if (gr) cudaGraphDestroy(gr);
      if (rc != FV_OK || ce != cudaSuccess || ie != cudaSuccess) {
        // capture not possible here: clear the capture's error and run directly
        cudaGetLastError();
        t->bwd_exec = nullptr;
        t->bwd_graph_off = true;
        const int rc2 = tape_backward_enqueue(t, dsn, dparams, dq0, s);
        if (rc2 != FV_OK) return rc2;
        FV_CUDA_TRY(cudaStreamSynchronize(s));
        return fvs::net_check(t->net);
      }
      t->bwd_dsn = dsn;
      t->bwd_dparams = dparams;
      t->bwd_dq0 = dq0;
    }
    FV_CUDA_TRY(cudaGraphLaunch(t->bwd_exec, s));
  }
  FV_CUDA_TRY(cudaStreamSynchronize(s));
  return fvs::net_check(t->net);
}

extern "C" int stencil_net_adam_step(fv_net* n, const float* grad, int step, double lr, double b1,
                                     double b2, double eps) {
  if (!n || !grad || step < 1) return fvh::fail(FV_EINVAL, "bad Adam arguments");
  const int np = snk::n_params(n->n.kind);
  if (!n->adam_m) {
    FV_CUDA_TRY(cudaMalloc(&n->adam_m, sizeof(float) * np));
    FV_CUDA_TRY(cudaMalloc(&n->adam_v, sizeof(float) * np));
    FV_CUDA_TRY(cudaMemsetAsync(n->adam_m, 0, sizeof(float) * np, n->stream));
    FV_CUDA_TRY(cudaMemsetAsync(n->adam_v, 0, sizeof(float) * np, n->stream));
  }
  const double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
  fvk::adam_kernel<<<(np + 255) / 256, 256, 0, n->stream>>>(
      n->n.params, grad, n->adam_m, n->adam_v, np, (float)lr, (float)b1, (float)b2,
      (float)eps, (float)c1, (float)c2);
  FV_CUDA_TRY(cudaGetLastError());
  FV_CUDA_TRY(snk::repack(n->n, n->stream));
  FV_CUDA_TRY(cudaStreamSynchronize(n->stream));
  return FV_OK;
}
