// fv_learned.cu — the learned-stencil SSP-RK2 step (shallow water).
//
// Each Runge-Kutta stage (Eq. 2.19) runs the CNN on the stage input to get the
// 36 normalised coefficients per cell (Section 2.5.3, fourth approach), then
// one fused stage kernel: face states from the coefficients of the face's
// owner cell (cell i owns faces i+1/2 in x and j+1/2 in y),
//   Q^L = wL0 Q_{i-1} + wL1 Q_i + wL2 Q_{i+1},  Q^R = wR0 Q_i + wR1 Q_{i+1} + wR2 Q_{i+2},
// replaced by the MUSCL-minmod states (Eq. 2.18) wherever a learned depth
// falls below h_min (positivity fallback); then the same HLL flux, flux
// divergence and RK combine as the plain step.
//
// The face-state network (Section 2.5.3, third approach) gives each cell the
// states on its four sides directly; its stage kernel pairs the east (north)
// state of one cell with the west (south) state of the next at every face
// and applies the same HLL flux, divergence and RK combine.
#include <cuda_runtime.h>

#include <vector>

#include "fv_common.cuh"
#include "fv_internal.h"
#include "fv_learned.cuh"
#include "stencil_net.cuh"

struct fv_learned_ws {
  float* w = nullptr;          // coefficients [B][36][plane]
  float* sides = nullptr;      // face-state network: side states [B][12][plane]
  float* hmin = nullptr;       // per member positivity threshold (device)
  snk::Acts acts;
};

namespace fvk {
namespace {

constexpr int TX = 64, TY = 16, SX = TX + 4, SY = TY + 4, NT = 256;
constexpr int C = 3;

constexpr int learned_smem_bytes() {
  return (C * (SY * SX + TY * (TX + 1) + (TY + 1) * TX) + 4 * (NT / 32)) * 4;
}

struct LArgs {
  const float* qin;
  const float* qn;
  float* qout;
  const float* w;      // [B][36][plane]
  const float* hmin;   // [B]
  Ctrl* ctrl;
  const DtParams* dp;
  int nx, ny;
  long long plane, member;
  float rdx, rdy, g;
  int hx, hy;          // ring of a subdomain: outside the CFL reduction
};

template <int STAGE>
__global__ void __launch_bounds__(NT) stage_learned_kernel(LArgs a) {
  extern __shared__ float smem[];
  float* sq = smem;
  float* sF = sq + C * SY * SX;
  float* sG = sF + C * TY * (TX + 1);
  unsigned* red = reinterpret_cast<unsigned*>(sG + C * (TY + 1) * TX);
  const int b = blockIdx.z;
  Ctrl* ctrl = a.ctrl + b;
  if (skip_if_done(ctrl)) return;
  const float dt = (float)ctrl->dt;
  const float hmin = a.hmin[b];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const float* qin = a.qin + b * a.member;
  const float* wb = a.w + (long long)b * 36 * a.plane;
  const int tid = threadIdx.x;

  for (int idx = tid; idx < C * SY * SX; idx += NT) {
    const int c = idx / (SY * SX);
    const int r = idx - c * (SY * SX);
    const int sy = r / SX, sx = r - sy * SX;
    const int gx = wrap(x0 - 2 + sx, a.nx), gy = wrap(y0 - 2 + sy, a.ny);
    sq[idx] = qin[c * a.plane + (long long)gy * a.nx + gx];
  }
  __syncthreads();

  for (int idx = tid; idx < TY * (TX + 1); idx += NT) {
    const int r = idx / (TX + 1), k = idx - r * (TX + 1);
    const int gy = y0 + r;
    if (gy >= a.ny) continue;
    const long long owner = (long long)gy * a.nx + wrap(x0 - 1 + k, a.nx);
    const float* row = sq + (r + 2) * SX + k;
    float m[C], s0[C], s1[C], p[C], wd[18], L[C], R[C], F[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float* rc = row + c * SY * SX;
      m[c] = rc[0]; s0[c] = rc[1]; s1[c] = rc[2]; p[c] = rc[3];
    }
#pragma unroll
    for (int j = 0; j < 18; ++j) wd[j] = wb[j * a.plane + owner];
    learned_face(m, s0, s1, p, wd, hmin, L, R);
    hll_swe<float>(L[0], L[1], L[2], R[0], R[1], R[2], a.g, F[0], F[1], F[2]);
#pragma unroll
    for (int c = 0; c < C; ++c) sF[(c * TY + r) * (TX + 1) + k] = F[c];
  }
  for (int idx = tid; idx < (TY + 1) * TX; idx += NT) {
    const int k = idx / TX, i = idx - k * TX;
    const int gx = x0 + i;
    if (gx >= a.nx) continue;
    const long long owner = (long long)wrap(y0 - 1 + k, a.ny) * a.nx + gx;
    const float* col = sq + k * SX + (i + 2);
    float m[C], s0[C], s1[C], p[C], wd[18], L[C], R[C], F[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float* cc = col + c * SY * SX;
      m[c] = cc[0]; s0[c] = cc[SX]; s1[c] = cc[2 * SX]; p[c] = cc[3 * SX];
    }
#pragma unroll
    for (int j = 0; j < 18; ++j) wd[j] = wb[(18 + j) * a.plane + owner];
    learned_face(m, s0, s1, p, wd, hmin, L, R);
    // rotated frame: normal momentum = hv
    hll_swe<float>(L[0], L[2], L[1], R[0], R[2], R[1], a.g, F[0], F[2], F[1]);
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
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float L = divergence<float>(sF[(c * TY + r) * (TX + 1) + i], sF[(c * TY + r) * (TX + 1) + i + 1],
                                        sG[(c * (TY + 1) + r) * TX + i], sG[(c * (TY + 1) + r + 1) * TX + i],
                                        a.rdx, a.rdy);
      const float q = sq[(c * SY + r + 2) * SX + i + 2];
      out[c] = STAGE == 1 ? rk_stage1<float>(q, dt, L) : rk_stage2<float>(qn[c * a.plane + off], q, 0.5f * dt, L);
      qout[c * a.plane + off] = out[c];
    }
    if (STAGE == 2) {
      unsigned bk = 0u;
      const float sp = cell_rate_swe(out[0], out[1], out[2], a.g, a.rdx, a.rdy, bk);
      const bool in = gx >= a.hx && gx < a.nx - a.hx && gy >= a.hy && gy < a.ny - a.hy;
      amax = in ? fmaxf(amax, sp) : amax;
      bad |= in ? bk : 0u;
    }
  }
  if (STAGE == 2) {
    block_reduce_max_or(amax, bad, red);
    if (tid == 0) publish_and_close(ctrl, a.dp, amax, bad, gridDim.x * gridDim.y, true);
  }
}

struct FArgs {
  const float* qin;
  const float* qn;
  float* qout;
  const float* sides;  // [B][12][plane], channel 3 side + var, sides W, E, S, N
  Ctrl* ctrl;
  const DtParams* dp;
  int nx, ny;
  long long plane, member;
  float rdx, rdy, g;
  int hx, hy;          // ring of a subdomain: outside the CFL reduction
};

enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };

constexpr int face_smem_bytes() { return (C * (TY * (TX + 1) + (TY + 1) * TX) + 4 * (NT / 32)) * 4; }

template <int STAGE>
__global__ void __launch_bounds__(NT) stage_face_kernel(FArgs a) {
  extern __shared__ float smem[];
  float* sF = smem;                          // [C][TY][TX+1] x-face fluxes
  float* sG = sF + C * TY * (TX + 1);        // [C][TY+1][TX] y-face fluxes
  unsigned* red = reinterpret_cast<unsigned*>(sG + C * (TY + 1) * TX);
  const int b = blockIdx.z;
  Ctrl* ctrl = a.ctrl + b;
  if (skip_if_done(ctrl)) return;
  const float dt = (float)ctrl->dt;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const float* sb = a.sides + (long long)b * 12 * a.plane;
  const int tid = threadIdx.x;

  // x face k of tile row r: between cells x0 - 1 + k (its east state) and
  // x0 + k (its west state), periodic
  for (int idx = tid; idx < TY * (TX + 1); idx += NT) {
    const int r = idx / (TX + 1), k = idx - r * (TX + 1);
    const int gy = y0 + r;
    if (gy >= a.ny || x0 + k > a.nx) continue;
    const long long row = (long long)gy * a.nx;
    const long long cl = row + wrap(x0 - 1 + k, a.nx), cr = row + wrap(x0 + k, a.nx);
    float L[C], R[C], F[C];
#pragma unroll
    for (int v = 0; v < C; ++v) {
      L[v] = sb[(3 * SIDE_E + v) * a.plane + cl];
      R[v] = sb[(3 * SIDE_W + v) * a.plane + cr];
    }
    hll_swe<float>(L[0], L[1], L[2], R[0], R[1], R[2], a.g, F[0], F[1], F[2]);
#pragma unroll
    for (int c = 0; c < C; ++c) sF[(c * TY + r) * (TX + 1) + k] = F[c];
  }
  // y face k of tile column i: between rows y0 - 1 + k (north state) and
  // y0 + k (south state)
  for (int idx = tid; idx < (TY + 1) * TX; idx += NT) {
    const int k = idx / TX, i = idx - k * TX;
    const int gx = x0 + i;
    if (gx >= a.nx || y0 + k > a.ny) continue;
    const long long cl = (long long)wrap(y0 - 1 + k, a.ny) * a.nx + gx;
    const long long cr = (long long)wrap(y0 + k, a.ny) * a.nx + gx;
    float L[C], R[C], F[C];
#pragma unroll
    for (int v = 0; v < C; ++v) {
      L[v] = sb[(3 * SIDE_N + v) * a.plane + cl];
      R[v] = sb[(3 * SIDE_S + v) * a.plane + cr];
    }
    // rotated frame: normal momentum = hv
    hll_swe<float>(L[0], L[2], L[1], R[0], R[2], R[1], a.g, F[0], F[2], F[1]);
#pragma unroll
    for (int c = 0; c < C; ++c) sG[(c * (TY + 1) + k) * TX + i] = F[c];
  }
  __syncthreads();

  float amax = 0.f;
  unsigned bad = 0u;
  const float* qin = a.qin + b * a.member;
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
      const float L = divergence<float>(sF[(c * TY + r) * (TX + 1) + i], sF[(c * TY + r) * (TX + 1) + i + 1],
                                        sG[(c * (TY + 1) + r) * TX + i], sG[(c * (TY + 1) + r + 1) * TX + i],
                                        a.rdx, a.rdy);
      const float q = qin[c * a.plane + off];
      out[c] = STAGE == 1 ? rk_stage1<float>(q, dt, L) : rk_stage2<float>(qn[c * a.plane + off], q, 0.5f * dt, L);
      qout[c * a.plane + off] = out[c];
    }
    if (STAGE == 2) {
      unsigned bk = 0u;
      const float sp = cell_rate_swe(out[0], out[1], out[2], a.g, a.rdx, a.rdy, bk);
      const bool in = gx >= a.hx && gx < a.nx - a.hx && gy >= a.hy && gy < a.ny - a.hy;
      amax = in ? fmaxf(amax, sp) : amax;
      bad |= in ? bk : 0u;
    }
  }
  if (STAGE == 2) {
    block_reduce_max_or(amax, bad, red);
    if (tid == 0) publish_and_close(ctrl, a.dp, amax, bad, gridDim.x * gridDim.y, true);
  }
}

template <int STAGE>
cudaError_t launch_face_t(const FArgs& a, const Geom& g, cudaStream_t s) {
  constexpr int smem = face_smem_bytes();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(stage_face_kernel<STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, g.B);
  stage_face_kernel<STAGE><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

// One SSP-RK2 stage of the face-state path from the side states of qin.
cudaError_t launch_stage_face(const Geom& g, int stage, const float* qin, const float* qn, float* qout,
                              const float* sides, Ctrl* ctrl, const DtParams* dp, cudaStream_t s) {
  FArgs a{qin, qn, qout, sides, ctrl, dp, g.nx, g.ny, g.plane(), g.member(),
          (float)(1.0 / g.dx), (float)(1.0 / g.dy), g.phys, g.hx, g.hy};
  return stage == 1 ? launch_face_t<1>(a, g, s) : launch_face_t<2>(a, g, s);
}

cudaError_t launch_stage_learned(const Geom& g, int stage, const float* qin, const float* qn,
                                 float* qout, const float* w, const float* hmin, Ctrl* ctrl,
                                 const DtParams* dp, cudaStream_t s) {
  constexpr int smem = learned_smem_bytes();
  LArgs a{qin, qn, qout, w, hmin, ctrl, dp, g.nx, g.ny, g.plane(), g.member(),
          (float)(1.0 / g.dx), (float)(1.0 / g.dy), g.phys, g.hx, g.hy};
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, g.B);
  if (stage == 1) {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(stage_learned_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    stage_learned_kernel<1><<<grid, NT, smem, s>>>(a);
  } else {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(stage_learned_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    stage_learned_kernel<2><<<grid, NT, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace fvk

namespace fvs {

static bool use_fused(const fv_state* s) {
  return s->learned_variant != FV_LEARNED_TWO_PASS && fvk::learned_fused_supported(s->g.nx, s->g.ny);
}

static bool is_face(const fv_net* net) { return net && net->n.kind == snk::NET_FACE; }

// Workspace of the face-state path: the side states and the CNN activations.
static int face_ws_ready(fv_state* s) {
  if (!snk::grid_supported(s->g.nx) || s->g.plane() % snk::TILE != 0)
    return fvh::fail(FV_EINVAL, "face-state step: nx must be 8, 16, 32, 64 or a multiple of 128, "
                                "and nx*ny a multiple of 128");
  const long long cells = (long long)s->g.B * s->g.plane();
  if (!s->lws) s->lws = new fv_learned_ws();
  cudaError_t e = cudaSuccess;
  if (!s->lws->sides) e = cudaMalloc(&s->lws->sides, sizeof(float) * snk::N_OUT_FACE * cells);
  if (e == cudaSuccess) e = snk::acts_reserve(s->lws->acts, cells);
  return e == cudaSuccess ? FV_OK : fvh::cuda_fail(e, "face-state workspace");
}

// Lazily create the learned workspace of a state: h_min = frac * (mean depth
// of the current state) per member (the mean depth is conserved by the
// scheme), and, for the two-pass path only, the coefficient buffer and the
// CNN activations.  The workspace may already exist without h_min when the
// state took face-state steps first.
static int learned_ws_ready(fv_state* s, float hmin_frac) {
  const bool fused = use_fused(s);
  if (!fused && (!snk::grid_supported(s->g.nx) || s->g.plane() % snk::TILE != 0))
    return fvh::fail(FV_EINVAL, "learned step: nx must be 8, 16, 32, 64 or a multiple of 128, "
                                "and nx*ny a multiple of 128");
  const long long cells = (long long)s->g.B * s->g.plane();
  if (!s->lws) s->lws = new fv_learned_ws();
  fv_learned_ws* w = s->lws;
  cudaError_t e = cudaSuccess;
  if (!fused && !w->w) {
    e = cudaMalloc(&w->w, sizeof(float) * 36 * cells);
    if (e == cudaSuccess) e = snk::acts_reserve(w->acts, cells);
    if (e != cudaSuccess) return fvh::cuda_fail(e, "learned workspace");
  }
  if (w->hmin) return FV_OK;
  float* hmin = nullptr;
  e = cudaMalloc(&hmin, sizeof(float) * s->g.B);
  if (e == cudaSuccess) e = fvk::launch_diagnostics(s->g, s->qA, s->diag_partials, s->diag_out, s->stream);
  std::vector<double> sums((size_t)s->g.B * (s->g.C + 1));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sums.data(), s->diag_out, sizeof(double) * sums.size(), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) {
    std::vector<float> hm(s->g.B);
    const double area = s->lx * s->ly;
    for (int b = 0; b < s->g.B; ++b) hm[b] = (float)(hmin_frac * sums[(size_t)b * (s->g.C + 1)] / area);
    e = cudaMemcpy(hmin, hm.data(), sizeof(float) * s->g.B, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaFree(hmin);
    return fvh::cuda_fail(e, "learned workspace");
  }
  w->hmin = hmin;
  return FV_OK;
}

int learned_prepare(fv_state* s, const fv_net* net) {
  if (s->flux != FV_FLUX_HLL || s->rk != 2)
    return fvh::fail(FV_EINVAL, "the learned step uses the HLL flux and SSP-RK2 (see fv_set_scheme)");
  if (s->bc != FV_BC_PERIODIC || s->zbed)
    return fvh::fail(FV_EINVAL, "the learned step runs on periodic flat-bed grids");
  if (is_face(net)) return face_ws_ready(s);
  return learned_ws_ready(s, s->hmin_frac);
}

cudaError_t enqueue_learned_stage(fv_state* s, const fv_net* net, int stage) {
  if (!s->lws) return cudaErrorNotReady;   // learned_prepare() must run first (host side)
  fv_learned_ws* w = s->lws;
  const int B = s->g.B, ny = s->g.ny, nx = s->g.nx;
  // stage 1: q^n (qA) -> q1 (qB); stage 2: q1 (qB), q^n (qA) -> q^{n+1} (qA)
  float* qin = stage == 1 ? s->qA : s->qB;
  const float* qn = stage == 1 ? nullptr : s->qA;
  float* qout = stage == 1 ? s->qB : s->qA;
  if (is_face(net)) {
    if (!w->sides) return cudaErrorNotReady;
    cudaError_t e = snk::forward_faces(net->n, qin, B, ny, nx, w->acts, w->sides, nullptr, s->stream);
    if (e != cudaSuccess) return e;
    return fvk::launch_stage_face(s->g, stage, qin, qn, qout, w->sides, s->ctrl, s->dp, s->stream);
  }
  if (!w->hmin) return cudaErrorNotReady;
  if (use_fused(s))
    return fvk::launch_learned_fused(s->g, stage, qin, qn, qout, net->n, w->hmin, s->ctrl, s->dp, s->stream);
  if (!w->w) return cudaErrorNotReady;
  cudaError_t e = snk::forward(net->n, qin, B, ny, nx, w->acts, w->w, nullptr, s->stream);
  if (e != cudaSuccess) return e;
  return fvk::launch_stage_learned(s->g, stage, qin, qn, qout, w->w, w->hmin, s->ctrl, s->dp, s->stream);
}

cudaError_t enqueue_learned_step(fv_state* s, const fv_net* net) {
  cudaError_t e = enqueue_learned_stage(s, net, 1);
  if (e != cudaSuccess) return e;
  return enqueue_learned_stage(s, net, 2);
}

int learned_set_hmin_values(fv_state* s, const double* hmin) {
  if (learned_hmin_fixed(s)) return fvh::fail(FV_EINVAL, "h_min is already fixed (a learned step was taken)");
  if (!s->lws) s->lws = new fv_learned_ws();
  std::vector<float> hm(s->g.B);
  for (int b = 0; b < s->g.B; ++b) {
    if (!(hmin[b] >= 0.0)) return fvh::fail(FV_EINVAL, "h_min must be >= 0");
    hm[b] = (float)hmin[b];
  }
  float* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(float) * s->g.B);
  if (e == cudaSuccess) e = cudaMemcpy(d, hm.data(), sizeof(float) * s->g.B, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return fvh::cuda_fail(e, "h_min values");
  }
  s->lws->hmin = d;
  return FV_OK;
}

bool learned_hmin_fixed(const fv_state* s) { return s->lws && s->lws->hmin; }

float* learned_hmin_ptr(fv_state* s) { return s->lws ? s->lws->hmin : nullptr; }

long long learned_ws_bytes(const fv_state* s) {
  if (!s->lws) return 0;
  const fv_learned_ws* w = s->lws;
  const long long cells = (long long)s->g.B * s->g.plane();
  long long b = 0;
  if (w->w) b += 36LL * 4 * cells;
  if (w->sides) b += (long long)snk::N_OUT_FACE * 4 * cells;
  if (w->hmin) b += 4LL * s->g.B;
  for (int l = 0; l < 3; ++l)
    if (w->acts.a[l]) b += 2LL * 32 * w->acts.cells;
  return b;
}

void learned_workspace_free(fv_state* s) {
  if (!s->lws) return;
  cudaFree(s->lws->w);
  cudaFree(s->lws->sides);
  cudaFree(s->lws->hmin);
  snk::acts_free(s->lws->acts);
  delete s->lws;
  s->lws = nullptr;
}

}  // namespace fvs
