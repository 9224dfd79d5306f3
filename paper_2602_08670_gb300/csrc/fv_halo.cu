// fv_halo.cu — subdomains of a block-decomposed grid.
//
// A grid of nx x ny cells split into px x py blocks is held as px * py states
// of (nx/px + 2 hx) x (ny/py + 2 hy) cells: each block's interior plus a ring
// of hx columns and hy rows that copies its periodic neighbours' cells.  The
// ring is what one Runge-Kutta stage reads beyond the interior: 2 cells for
// MUSCL-minmod (Eq. 2.18), 5 for the learned stencils (the CNN's four 3x3
// layers reach 4 cells beyond the coefficients of the two faces of a cell,
// and those faces' stencils reach 2), rounded up to 6 to keep rows 16-byte
// aligned.  Every stage reads a ring refreshed after the previous stage; the
// stage kernels compute the ring cells too (from their own periodic wrap, so
// with wrong neighbours), and those values are overwritten by the next
// refresh.  The CFL reduction, the health bits and the diagnostics cover the
// interior only, and the next dt is the minimum over the subdomains, so the
// interiors evolve exactly as the undecomposed grid.
//
// Here: the ring of every subdomain of one process is filled in one kernel
// straight from its neighbours' interiors (several subdomains on one GPU);
// ring strips are packed to / unpacked from contiguous buffers for an
// exchange between processes (in x first over the interior rows, then in y
// over the full width, which carries the corners); the per-member dt is
// reduced to its minimum over the subdomains.
#include <cuda_runtime.h>

#include <vector>

#include "fv_common.cuh"
#include "fv_internal.h"

namespace {

constexpr int MAX_SUB = 64;

struct SubTable {
  float* q[MAX_SUB];
};

struct CtrlTable {
  fvk::Ctrl* c[MAX_SUB];
};

// Ring cell j (0 <= j < ring) of a (nxs + 2 hx) x (nys + 2 hy) subdomain:
// south rows, north rows, then the west and east columns of the interior rows.
__device__ __forceinline__ void ring_cell(long long j, int nxs, int nys, int hx, int hy, int& xe, int& ye) {
  const int nxe = nxs + 2 * hx;
  const long long rows = (long long)hy * nxe;
  if (j < rows) {
    ye = (int)(j / nxe);
    xe = (int)(j - (long long)ye * nxe);
    return;
  }
  j -= rows;
  if (j < rows) {
    ye = nys + hy + (int)(j / nxe);
    xe = (int)(j - (long long)(ye - nys - hy) * nxe);
    return;
  }
  j -= rows;
  const long long cols = (long long)hx * nys;
  const bool east = j >= cols;
  if (east) j -= cols;
  ye = hy + (int)(j / hx);
  const int c = (int)(j - (long long)(ye - hy) * hx);
  xe = east ? nxs + hx + c : c;
}

// Fill the ring of every subdomain (k = iy * px + ix) from the interiors of
// the subdomains that own those cells on the periodic px nxs x py nys grid.
// Reads interiors, writes rings: no cell is both.
__global__ void halo_fill_kernel(SubTable t, int px, int py, int nxs, int nys, int hx, int hy,
                                 long long planes) {
  const int nxe = nxs + 2 * hx, nye = nys + 2 * hy;
  const long long ring = 2LL * hy * nxe + 2LL * hx * nys;
  const long long plane = (long long)nxe * nye;
  const long long per_sub = ring * planes;
  const long long total = per_sub * px * py;
  const int NX = px * nxs, NY = py * nys;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / per_sub);
    const long long r = i - (long long)k * per_sub;
    const long long p = r / ring;
    int xe, ye;
    ring_cell(r - p * ring, nxs, nys, hx, hy, xe, ye);
    const int ix = k % px, iy = k / px;
    int gx = ix * nxs + xe - hx, gy = iy * nys + ye - hy;
    gx = gx < 0 ? gx + NX : (gx >= NX ? gx - NX : gx);
    gy = gy < 0 ? gy + NY : (gy >= NY ? gy - NY : gy);
    const int sx = gx / nxs, sy = gy / nys;
    const int lx = gx - sx * nxs + hx, ly = gy - sy * nys + hy;
    t.q[k][p * plane + (long long)ye * nxe + xe] = t.q[sy * px + sx][p * plane + (long long)ly * nxe + lx];
  }
}

// Copy the w x h window at (x0, y0) of every plane of a [planes][ny][nx]
// buffer to a contiguous [planes][h][w] buffer (pack) or back (unpack).
__global__ void strip_copy_kernel(float* grid, float* strip, int nx, long long plane, int x0, int y0, int w,
                                  int h, long long planes, bool pack) {
  const long long per = (long long)w * h;
  const long long total = per * planes;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / per;
    const long long r = i - p * per;
    const int y = (int)(r / w), x = (int)(r - (long long)y * w);
    float* g = grid + p * plane + (long long)(y0 + y) * nx + x0 + x;
    if (pack) strip[i] = *g;
    else *g = strip[i];
  }
}

// Per member: the smallest pending dt and the largest Courant rate over the
// subdomains, written back to all of them.
__global__ void dt_min_kernel(CtrlTable t, int n, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double dt = t.c[0][b].dt, am = t.c[0][b].amax_last;
  for (int k = 1; k < n; ++k) {
    dt = fmin(dt, t.c[k][b].dt);
    am = fmax(am, t.c[k][b].amax_last);
  }
  for (int k = 0; k < n; ++k) {
    t.c[k][b].dt = dt;
    t.c[k][b].amax_last = am;
  }
}

unsigned grid_blocks(long long work) {
  long long b = (work + 255) / 256;
  if (b > 4096) b = 4096;
  return (unsigned)(b > 0 ? b : 1);
}

// Subdomains of one decomposition: same equations, batch and extended shape.
int check_subs(fv_state* const* subs, int n) {
  if (!subs || n < 1 || n > MAX_SUB) return fvh::fail(FV_EINVAL, "1 to 64 subdomain states");
  for (int k = 0; k < n; ++k) {
    if (!subs[k]) return fvh::fail(FV_EINVAL, "null subdomain state");
    const fvk::Geom &a = subs[0]->g, &b = subs[k]->g;
    if (b.eq != a.eq || b.B != a.B || b.C != a.C || b.nx != a.nx || b.ny != a.ny || b.hx != a.hx || b.hy != a.hy)
      return fvh::fail(FV_EINVAL, "subdomain states differ in equations, batch, shape or ring");
  }
  return FV_OK;
}

// Order subs[0]'s stream after all others (fork-join through their events),
// and the others after what is then enqueued on subs[0]'s stream.
cudaError_t join_streams(fv_state* const* subs, int n) {
  for (int k = 0; k < n; ++k) {
    cudaError_t e = fvs::enter(subs[k]);
    if (e != cudaSuccess) return e;
  }
  for (int k = 1; k < n; ++k) {
    if (subs[k]->stream == subs[0]->stream) continue;
    cudaError_t e = cudaEventRecord(subs[k]->ev, subs[k]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(subs[0]->stream, subs[k]->ev, 0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t fork_streams(fv_state* const* subs, int n) {
  for (int k = 1; k < n; ++k) {
    if (subs[k]->stream == subs[0]->stream) continue;
    cudaError_t e = cudaEventRecord(subs[0]->ev, subs[0]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(subs[k]->stream, subs[0]->ev, 0);
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k < n; ++k) {
    cudaError_t e = fvs::leave(subs[k]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

float* buffer_of(fv_state* s, int buf) { return buf == 0 ? s->qA : s->qB; }

}  // namespace

extern "C" int fv_set_halo(fv_state* s, int hx, int hy) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (s->g.eq == fvk::SPHERE) return fvh::fail(FV_EINVAL, "a sphere state has no subdomains");
  if (hx < 0 || hy < 0 || 4 * hx > s->g.nx || 4 * hy > s->g.ny)
    return fvh::fail(FV_EINVAL, "fv_set_halo: the interior must be at least as wide as the two rings");
  if (s->bc != FV_BC_PERIODIC || s->zbed)
    return fvh::fail(FV_EINVAL, "fv_set_halo: subdomains of periodic flat-bed grids only");
  s->g.hx = hx;
  s->g.hy = hy;
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);   // its launches carry the old interior
    s->graph = nullptr;
  }
  FV_CUDA_TRY(fvs::enter(s));
  FV_CUDA_TRY(fvs::wavespeed_init(s));   // dt of the interior
  FV_CUDA_TRY(fvs::leave(s));
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return fvs::check_health(s);
}

extern "C" int fv_enqueue_stage(fv_state* s, const fv_net* net, int stage) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (stage != 1 && stage != 2) return fvh::fail(FV_EINVAL, "stage is 1 or 2");
  if (s->g.eq == fvk::SPHERE) return fvh::fail(FV_EINVAL, "fv_enqueue_stage: planar states only");
  if (net) {
    if (s->g.eq != fvk::SWE) return fvh::fail(FV_EINVAL, "learned step is SWE only");
    int rc = fvs::learned_prepare(s, net);
    if (rc != FV_OK) return rc;
  } else if (s->flux != FV_FLUX_HLL || s->rk != 2 || s->bc != FV_BC_PERIODIC || s->zbed) {
    return fvh::fail(FV_EINVAL, "fv_enqueue_stage: HLL, SSP-RK2, periodic flat bed");
  }
  FV_CUDA_TRY(fvs::enter(s));
  FV_CUDA_TRY(net ? fvs::enqueue_learned_stage(s, net, stage) : fvs::enqueue_plain_stage(s, stage));
  FV_CUDA_TRY(fvs::leave(s));
  return FV_OK;
}

extern "C" int fv_halo_exchange(fv_state* const* subs, int px, int py, int buf) {
  if (px < 1 || py < 1) return fvh::fail(FV_EINVAL, "px, py >= 1");
  int rc = check_subs(subs, px * py);
  if (rc != FV_OK) return rc;
  if (buf != 0 && buf != 1) return fvh::fail(FV_EINVAL, "buf is 0 (q^n) or 1 (stage output)");
  const fvk::Geom& g = subs[0]->g;
  if ((px > 1 && g.hx == 0) || (py > 1 && g.hy == 0))
    return fvh::fail(FV_EINVAL, "fv_halo_exchange: a split direction needs a ring (fv_set_halo)");
  const int n = px * py;
  SubTable t{};
  for (int k = 0; k < n; ++k) t.q[k] = buffer_of(subs[k], buf);
  const int nxs = g.nx - 2 * g.hx, nys = g.ny - 2 * g.hy;
  const long long planes = (long long)g.B * g.C;
  const long long ring = 2LL * g.hy * g.nx + 2LL * g.hx * nys;
  FV_CUDA_TRY(join_streams(subs, n));
  if (ring > 0) {
    halo_fill_kernel<<<grid_blocks(ring * planes * n), 256, 0, subs[0]->stream>>>(t, px, py, nxs, nys, g.hx,
                                                                                  g.hy, planes);
    FV_CUDA_TRY(cudaGetLastError());
  }
  FV_CUDA_TRY(fork_streams(subs, n));
  return FV_OK;
}

extern "C" int fv_reduce_dt(fv_state* const* subs, int n) {
  int rc = check_subs(subs, n);
  if (rc != FV_OK) return rc;
  CtrlTable t{};
  for (int k = 0; k < n; ++k) t.c[k] = subs[k]->ctrl;
  const int B = subs[0]->g.B;
  FV_CUDA_TRY(join_streams(subs, n));
  dt_min_kernel<<<(B + 127) / 128, 128, 0, subs[0]->stream>>>(t, n, B);
  FV_CUDA_TRY(cudaGetLastError());
  FV_CUDA_TRY(fork_streams(subs, n));
  return FV_OK;
}

namespace {

// Window of side `side` (0 W, 1 E, 2 S, 3 N): the interior strip a neighbour
// needs (pack) or the ring strip it fills (unpack).
void side_window(const fvk::Geom& g, int side, bool pack, int& x0, int& y0, int& w, int& h) {
  const int nxs = g.nx - 2 * g.hx, nys = g.ny - 2 * g.hy;
  if (side < 2) {                  // columns, interior rows only
    w = g.hx;
    h = nys;
    y0 = g.hy;
    if (pack) x0 = side == 0 ? g.hx : nxs;
    else x0 = side == 0 ? 0 : nxs + g.hx;
  } else {                         // rows, the full width (rings included: corners)
    w = g.nx;
    h = g.hy;
    x0 = 0;
    if (pack) y0 = side == 2 ? g.hy : nys;
    else y0 = side == 2 ? 0 : nys + g.hy;
  }
}

int strip_io(fv_state* s, int buf, int side, float* strip, bool pack) {
  if (!s || !strip) return fvh::fail(FV_EINVAL, "null argument");
  if (buf != 0 && buf != 1) return fvh::fail(FV_EINVAL, "buf is 0 (q^n) or 1 (stage output)");
  if (side < 0 || side > 3) return fvh::fail(FV_EINVAL, "side is 0 (W), 1 (E), 2 (S) or 3 (N)");
  int x0, y0, w, h;
  side_window(s->g, side, pack, x0, y0, w, h);
  if (w == 0 || h == 0) return fvh::fail(FV_EINVAL, "no ring on that side (fv_set_halo)");
  const long long planes = (long long)s->g.B * s->g.C;
  FV_CUDA_TRY(fvs::enter(s));
  strip_copy_kernel<<<grid_blocks((long long)w * h * planes), 256, 0, s->stream>>>(
      buffer_of(s, buf), strip, s->g.nx, s->g.plane(), x0, y0, w, h, planes, pack);
  FV_CUDA_TRY(cudaGetLastError());
  FV_CUDA_TRY(fvs::leave(s));
  return FV_OK;
}

}  // namespace

extern "C" int fv_halo_pack(fv_state* s, int buf, int side, float* dst) {
  return strip_io(s, buf, side, dst, true);
}

extern "C" int fv_halo_unpack(fv_state* s, int buf, int side, const float* src) {
  return strip_io(s, buf, side, const_cast<float*>(src), false);
}

extern "C" int fv_halo_strip_floats(const fv_state* s, int side, long long* n) {
  if (!s || !n || side < 0 || side > 3) return fvh::fail(FV_EINVAL, "bad arguments");
  int x0, y0, w, h;
  side_window(s->g, side, true, x0, y0, w, h);
  *n = (long long)w * h * s->g.B * s->g.C;
  return FV_OK;
}

extern "C" int fv_set_dt(fv_state* s, const double* dt) {
  if (!s || !dt) return fvh::fail(FV_EINVAL, "null argument");
  for (int b = 0; b < s->g.B; ++b)
    if (!(dt[b] >= 0.0)) return fvh::fail(FV_EINVAL, "dt must be >= 0");
  std::vector<fvk::Ctrl> c(s->g.B);
  FV_CUDA_TRY(fvs::enter(s));
  FV_CUDA_TRY(cudaMemcpyAsync(c.data(), s->ctrl, sizeof(fvk::Ctrl) * s->g.B, cudaMemcpyDeviceToHost, s->stream));
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  for (int b = 0; b < s->g.B; ++b) c[b].dt = dt[b];
  FV_CUDA_TRY(cudaMemcpyAsync(s->ctrl, c.data(), sizeof(fvk::Ctrl) * s->g.B, cudaMemcpyHostToDevice, s->stream));
  FV_CUDA_TRY(fvs::leave(s));
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return FV_OK;
}

extern "C" int fv_set_learned_hmin_values(fv_state* s, const double* hmin) {
  if (!s || !hmin) return fvh::fail(FV_EINVAL, "null argument");
  return fvs::learned_set_hmin_values(s, hmin);
}
