// fv_state.cu — C ABI of the plain finite-volume state: creation, stepping,
// graph-captured rollouts, state access, health and FP64 diagnostics.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "fv_common.cuh"
#include "fv_internal.h"
#include "fv_kernels.h"
#include "stencil_net.cuh"

// ---------------------------------------------------------------------------
// Error reporting
// ---------------------------------------------------------------------------
namespace fvh {
static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? FV_ENOMEM : FV_ECUDA;
}
}  // namespace fvh

extern "C" const char* fv_last_error(void) { return fvh::g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// Helpers
// ---------------------------------------------------------------------------
namespace {

cudaMemcpyKind kind_to_device(int loc) {
  return loc == FV_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_from_device(int loc) {
  return loc == FV_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

int create_state(const fv_grid* grid, int eq, double phys, double cfl, int dt_mode,
                 double dt_fixed, const float* q0, int q0_loc, void* stream, fv_state** out) {
  if (!grid || !q0 || !out) return fvh::fail(FV_EINVAL, "null argument");
  *out = nullptr;
  if (grid->nx < 1 || grid->ny < 1 || grid->batch < 1)
    return fvh::fail(FV_EINVAL, "grid sizes must be >= 1");
  if (!(grid->lx > 0) || !(grid->ly > 0)) return fvh::fail(FV_EINVAL, "domain lengths must be > 0");
  if (dt_mode < FV_DT_ADAPTIVE || dt_mode > FV_DT_REPLAY) return fvh::fail(FV_EINVAL, "bad dt_mode");
  if (dt_mode == FV_DT_ADAPTIVE && !(cfl > 0)) return fvh::fail(FV_EINVAL, "cfl must be > 0");
  if (dt_mode == FV_DT_FIXED && !(dt_fixed > 0)) return fvh::fail(FV_EINVAL, "dt_fixed must be > 0");
  if (q0_loc != FV_HOST && q0_loc != FV_DEVICE) return fvh::fail(FV_EINVAL, "bad q0 location");
  if (eq == fvk::SWE && !(phys > 0)) return fvh::fail(FV_EINVAL, "g must be > 0");
  if (eq == fvk::EULER && !(phys > 1)) return fvh::fail(FV_EINVAL, "gamma must be > 1");

  fv_state* s = new fv_state();
  s->g.nx = grid->nx;
  s->g.ny = grid->ny;
  s->g.B = grid->batch;
  s->g.C = eq == fvk::SWE ? 3 : 4;
  s->g.eq = eq;
  s->g.dx = grid->lx / grid->nx;
  s->g.dy = grid->ly / grid->ny;
  s->g.phys = (float)phys;
  s->g.phys_d = phys;
  s->lx = grid->lx;
  s->ly = grid->ly;
  s->dt_mode = dt_mode;
  s->user_stream = (cudaStream_t)stream;
  int rc = fvs::state_alloc(s);
  if (rc != FV_OK) {
    fvs::state_free(s);
    return rc;
  }
  const size_t bytes = (size_t)s->g.member() * s->g.B * sizeof(float);
  cudaError_t e = fvs::enter(s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->qA, q0, bytes, kind_to_device(q0_loc), s->stream);
  if (e == cudaSuccess) {
    fvk::DtParams dp{};
    dp.mode = dt_mode;
    dp.cfl = cfl;
    dp.dt_fixed = dt_fixed;
    dp.replay = nullptr;
    dp.replay_len = 0;
    s->dp_host = dp;
    e = cudaMemcpyAsync(s->dp, &s->dp_host, sizeof(fvk::DtParams), cudaMemcpyHostToDevice,
                        s->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(s->ctrl, 0, sizeof(fvk::Ctrl) * s->g.B, s->stream);
  // sphere states set their dt once their metrics exist (sphere_init)
  if (e == cudaSuccess && eq != fvk::SPHERE) e = fvk::launch_wavespeed_init(s->g, s->qA, s->ctrl, s->dp, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    fvs::state_free(s);
    return fvh::cuda_fail(e, "state initialisation");
  }
  *out = s;
  return FV_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Internal state management (shared with the learned-path translation unit)
// ---------------------------------------------------------------------------
namespace fvs {

// A caller stream that is a real stream object is used directly; the legacy
// and per-thread default streams (which cannot be captured into graphs) get a
// library-owned stream ordered against them with events.
static bool is_default_stream(cudaStream_t st) {
  return st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
}

int state_alloc(fv_state* s) {
  const size_t bytes = (size_t)s->g.member() * s->g.B * sizeof(float);
  cudaError_t e = cudaSuccess;
  if (!is_default_stream(s->user_stream)) {
    s->stream = s->user_stream;
    s->own_stream = false;
  } else {
    e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fvh::cuda_fail(e, "cudaStreamCreate");
    s->own_stream = true;
  }
  if ((e = cudaMalloc(&s->qA, bytes)) != cudaSuccess) return fvh::cuda_fail(e, "cudaMalloc(q)");
  if ((e = cudaMalloc(&s->qB, bytes)) != cudaSuccess) return fvh::cuda_fail(e, "cudaMalloc(q1)");
  if ((e = cudaMalloc(&s->ctrl, sizeof(fvk::Ctrl) * s->g.B)) != cudaSuccess)
    return fvh::cuda_fail(e, "cudaMalloc(ctrl)");
  if ((e = cudaMalloc(&s->dp, sizeof(fvk::DtParams))) != cudaSuccess)
    return fvh::cuda_fail(e, "cudaMalloc(dt params)");
  const long long np = fvk::diag_partials_size(s->g);
  if ((e = cudaMalloc(&s->diag_partials, sizeof(double) * np)) != cudaSuccess)
    return fvh::cuda_fail(e, "cudaMalloc(diag)");
  if ((e = cudaMalloc(&s->diag_out, sizeof(double) * s->g.B * (s->g.C + 1))) != cudaSuccess)
    return fvh::cuda_fail(e, "cudaMalloc(diag)");
  if ((e = cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming)) != cudaSuccess)
    return fvh::cuda_fail(e, "cudaEventCreate");
  return FV_OK;
}

long long state_device_bytes(const fv_state* s) {
  const long long q = (long long)s->g.member() * s->g.B * (long long)sizeof(float);
  long long b = 2 * q + (s->qC ? q : 0);
  b += (long long)sizeof(fvk::Ctrl) * s->g.B + (long long)sizeof(fvk::DtParams);
  b += (long long)sizeof(double) * (fvk::diag_partials_size(s->g) + (long long)s->g.B * (s->g.C + 1));
  return b + learned_ws_bytes(s);
}

void state_free(fv_state* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  cudaFree(s->qA);
  cudaFree(s->qB);
  cudaFree(s->qC);
  cudaFree(s->zbed);
  cudaFree(s->ctrl);
  cudaFree(s->dp);
  cudaFree(s->replay);
  cudaFree(s->diag_partials);
  cudaFree(s->diag_out);
  cudaFree(s->sphere);
  learned_workspace_free(s);
  if (s->ev) cudaEventDestroy(s->ev);
  if (s->stream && s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
}

// Order the state's stream after work already enqueued on the caller's stream.
cudaError_t enter(fv_state* s) {
  if (!s->own_stream || !s->user_stream) return cudaSuccess;
  cudaError_t e = cudaEventRecord(s->ev, s->user_stream);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(s->stream, s->ev, 0);
}

// Order later work on the caller's stream after what this call enqueued.
cudaError_t leave(fv_state* s) {
  if (!s->own_stream || !s->user_stream) return cudaSuccess;
  cudaError_t e = cudaEventRecord(s->ev, s->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(s->user_stream, s->ev, 0);
}

cudaError_t wavespeed_init(fv_state* s) {
  if (s->g.eq == fvk::SPHERE) return fvk::launch_sphere_wavespeed(s->g, s->qA, s->sphere, s->ctrl, s->dp, s->stream);
  return fvk::launch_wavespeed_init(s->g, s->qA, s->ctrl, s->dp, s->stream);
}

cudaError_t enqueue_plain_step(fv_state* s) {
  if (s->g.eq == fvk::SPHERE)
    return fvk::enqueue_sphere_step(s->g, s->flux, s->qA, s->qB, s->sphere, s->omega, s->ctrl, s->dp, s->stream);
  if (s->flux != FV_FLUX_HLL || s->rk != 2 || s->bc != FV_BC_PERIODIC || s->zbed)
    return fvk::enqueue_scheme_step(s->g, s->flux, s->rk, s->qA, s->qB, s->qC, s->ctrl, s->dp, s->stream,
                                    s->variant, s->bc, s->zbed);
  cudaError_t e = fvk::launch_stage_minmod(s->g, 1, s->qA, nullptr, s->qB, s->ctrl, s->dp,
                                           s->stream, s->variant);
  if (e != cudaSuccess) return e;
  return fvk::launch_stage_minmod(s->g, 2, s->qB, s->qA, s->qA, s->ctrl, s->dp, s->stream,
                                  s->variant);
}

cudaError_t enqueue_plain_stage(fv_state* s, int stage) {
  if (stage == 1)
    return fvk::launch_stage_minmod(s->g, 1, s->qA, nullptr, s->qB, s->ctrl, s->dp, s->stream, s->variant);
  return fvk::launch_stage_minmod(s->g, 2, s->qB, s->qA, s->qA, s->ctrl, s->dp, s->stream, s->variant);
}

cudaError_t enqueue_step(fv_state* s, const fv_net* net) {
  if (net) return enqueue_learned_step(s, net);
  return enqueue_plain_step(s);
}

int check_health(fv_state* s) {
  std::vector<fvk::Ctrl> c(s->g.B);
  cudaError_t e = cudaMemcpy(c.data(), s->ctrl, sizeof(fvk::Ctrl) * s->g.B, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fvh::cuda_fail(e, "reading health");
  for (int b = 0; b < s->g.B; ++b) {
    if (c[b].health) {
      char buf[160];
      snprintf(buf, sizeof buf, "member %d unstable: health bits 0x%x at step %lld (t=%.6g)", b,
               c[b].health, c[b].step, c[b].t);
      return fvh::fail(FV_EUNSTABLE, buf);
    }
  }
  return FV_OK;
}

}  // namespace fvs

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int swe_init(const fv_grid* grid, const fv_swe_params* p, const float* q0, int q0_loc,
                        void* stream, fv_state** out) {
  if (!p) return fvh::fail(FV_EINVAL, "null params");
  return create_state(grid, fvk::SWE, p->g, p->cfl, p->dt_mode, p->dt_fixed, q0, q0_loc, stream, out);
}

extern "C" int euler_init(const fv_grid* grid, const fv_euler_params* p, const float* q0,
                          int q0_loc, void* stream, fv_state** out) {
  if (!p) return fvh::fail(FV_EINVAL, "null params");
  return create_state(grid, fvk::EULER, p->gamma, p->cfl, p->dt_mode, p->dt_fixed, q0, q0_loc,
                      stream, out);
}

extern "C" int sphere_init(int nx, int ny, int batch, const fv_sphere_params* p, const float* q0, int q0_loc,
                           void* stream, fv_state** out) {
  if (!p || !out) return fvh::fail(FV_EINVAL, "null argument");
  if (ny < 2 || nx != 2 * ny) return fvh::fail(FV_EINVAL, "sphere grid: nx must be 2 ny and ny >= 2");
  if (!(p->g > 0.0)) return fvh::fail(FV_EINVAL, "g must be > 0");
  if (!(fabs(p->omega) < 1e30)) return fvh::fail(FV_EINVAL, "omega must be finite");
  fv_grid grid{nx, ny, batch, 4.0, 2.0};
  int rc = create_state(&grid, fvk::SPHERE, p->g, p->cfl, p->dt_mode, p->dt_fixed, q0, q0_loc, stream, out);
  if (rc != FV_OK) return rc;
  fv_state* s = *out;
  s->omega = (float)p->omega;
  cudaError_t e = cudaMalloc(&s->sphere, sizeof(float) * fvk::sphere_metric_floats(nx, ny));
  if (e == cudaSuccess) e = fvk::launch_sphere_metrics(s->sphere, nx, ny, s->stream);
  if (e == cudaSuccess) e = fvs::wavespeed_init(s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    fvs::state_free(s);
    *out = nullptr;
    return fvh::cuda_fail(e, "sphere_init");
  }
  return FV_OK;
}

extern "C" int sphere_get_cells(const fv_state* s, float* centres, float* areas, int loc) {
  if (!s || (!centres && !areas)) return fvh::fail(FV_EINVAL, "null argument");
  if (s->g.eq != fvk::SPHERE) return fvh::fail(FV_EINVAL, "not a sphere state");
  const int nx = s->g.nx, ny = s->g.ny;
  const cudaMemcpyKind k = loc == FV_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (centres)
    FV_CUDA_TRY(cudaMemcpy(centres, s->sphere + fvk::sphere_centre_offset(nx, ny), sizeof(float) * 3 * s->g.plane(), k));
  if (areas)
    FV_CUDA_TRY(cudaMemcpy(areas, s->sphere + fvk::sphere_area_offset(nx, ny), sizeof(float) * s->g.plane(), k));
  return FV_OK;
}

extern "C" int fv_destroy_state(fv_state* s) {
  fvs::state_free(s);
  return FV_OK;
}

extern "C" int fv_set_replay_dt(fv_state* s, const double* dts, long n) {
  if (!s || !dts || n < 1) return fvh::fail(FV_EINVAL, "bad replay arguments");
  if (n > 0x7fffffffL) return fvh::fail(FV_EINVAL, "replay sequence too long");
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  cudaFree(s->replay);
  s->replay = nullptr;
  FV_CUDA_TRY(cudaMalloc(&s->replay, sizeof(double) * n));
  FV_CUDA_TRY(cudaMemcpy(s->replay, dts, sizeof(double) * n, cudaMemcpyHostToDevice));
  s->dp_host.replay = s->replay;
  s->dp_host.replay_len = (int)n;
  FV_CUDA_TRY(cudaMemcpy(s->dp, &s->dp_host, sizeof(fvk::DtParams), cudaMemcpyHostToDevice));
  // the pending dt of a REPLAY state is the replay value of its current step
  if (s->dt_mode == FV_DT_REPLAY) FV_CUDA_TRY(fvs::wavespeed_init(s));
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return FV_OK;
}

extern "C" int fv_step(fv_state* s, const fv_net* net) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (net && s->g.eq != fvk::SWE) return fvh::fail(FV_EINVAL, "learned step is SWE only");
  if (net) {
    int rc = fvs::learned_prepare(s, net);
    if (rc != FV_OK) return rc;
  }
  FV_CUDA_TRY(fvs::enter(s));
  FV_CUDA_TRY(fvs::enqueue_step(s, net));
  FV_CUDA_TRY(fvs::leave(s));
  return FV_OK;
}

extern "C" int fv_sync(fv_state* s) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return fvs::check_health(s);
}

namespace {

// Enqueue nsteps steps: whole chunks replay one captured graph, the rest are
// launched directly.  If snaps is set, the state after every chunk is copied
// out.  Asynchronous.
int enqueue_steps(fv_state* s, const fv_net* net, long nsteps, long chunk, float* snaps,
                  int snaps_loc) {
  const size_t state_bytes = (size_t)s->g.member() * s->g.B * sizeof(float);
  long done = 0, snap_idx = 0;
  while (done < nsteps) {
    const long k = (nsteps - done) < chunk ? (nsteps - done) : chunk;
    if (k == chunk && chunk > 1) {
      if (!s->graph || s->graph_steps != chunk || s->graph_net != net) {
        if (s->graph) cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
        cudaGraph_t gr;
        FV_CUDA_TRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = cudaSuccess;
        for (long i = 0; i < chunk && ce == cudaSuccess; ++i) ce = fvs::enqueue_step(s, net);
        cudaError_t ee = cudaStreamEndCapture(s->stream, &gr);
        if (ce != cudaSuccess) return fvh::cuda_fail(ce, "capturing the step");
        if (ee != cudaSuccess) return fvh::cuda_fail(ee, "cudaStreamEndCapture");
        ee = cudaGraphInstantiate(&s->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (ee != cudaSuccess) return fvh::cuda_fail(ee, "cudaGraphInstantiate");
        s->graph_steps = chunk;
        s->graph_net = net;
      }
      FV_CUDA_TRY(cudaGraphLaunch(s->graph, s->stream));
    } else {
      for (long i = 0; i < k; ++i) FV_CUDA_TRY(fvs::enqueue_step(s, net));
    }
    done += k;
    if (snaps && k == chunk) {
      FV_CUDA_TRY(cudaMemcpyAsync((char*)snaps + state_bytes * snap_idx, s->qA, state_bytes,
                                  kind_from_device(snaps_loc), s->stream));
      ++snap_idx;
    }
  }
  return FV_OK;
}

}  // namespace

extern "C" int fv_enqueue_steps(fv_state* s, const fv_net* net, long nsteps) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (nsteps < 0) return fvh::fail(FV_EINVAL, "nsteps < 0");
  if (net && s->g.eq != fvk::SWE) return fvh::fail(FV_EINVAL, "learned step is SWE only");
  if (net) {
    int rc = fvs::learned_prepare(s, net);
    if (rc != FV_OK) return rc;
  }
  FV_CUDA_TRY(fvs::enter(s));
  const long chunk = nsteps < 32 ? (nsteps > 0 ? nsteps : 1) : 32;
  int rc = enqueue_steps(s, net, nsteps, chunk, nullptr, FV_DEVICE);
  if (rc != FV_OK) return rc;
  FV_CUDA_TRY(fvs::leave(s));
  return FV_OK;
}

extern "C" int fv_rollout(fv_state* s, const fv_net* net, long nsteps, double t_end, float* snaps,
                          int snaps_loc, int snap_every, double* t_out) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (nsteps < 0) return fvh::fail(FV_EINVAL, "nsteps < 0");
  if (net && s->g.eq != fvk::SWE) return fvh::fail(FV_EINVAL, "learned step is SWE only");
  if (snaps && snap_every <= 0) return fvh::fail(FV_EINVAL, "snap_every must be > 0 with snaps");
  if (net) {
    int rc = fvs::learned_prepare(s, net);
    if (rc != FV_OK) return rc;
  }
  FV_CUDA_TRY(fvs::enter(s));
  FV_CUDA_TRY(fvk::launch_set_t_end(s->ctrl, s->g.B, t_end, s->stream));
  const long chunk = snaps ? snap_every : (nsteps < 32 ? (nsteps > 0 ? nsteps : 1) : 32);
  int rc = enqueue_steps(s, net, nsteps, chunk, snaps, snaps_loc);
  if (rc != FV_OK) return rc;
  FV_CUDA_TRY(fvs::leave(s));
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (t_out) {
    std::vector<fvk::Ctrl> c(s->g.B);
    FV_CUDA_TRY(cudaMemcpy(c.data(), s->ctrl, sizeof(fvk::Ctrl) * s->g.B, cudaMemcpyDeviceToHost));
    for (int b = 0; b < s->g.B; ++b) t_out[b] = c[b].t;
  }
  if (net) {
    int rc = fvs::net_check(net);
    if (rc != FV_OK) return rc;
  }
  return fvs::check_health(s);
}

extern "C" int fv_get_state(const fv_state* cs, float* dst, int dst_loc) {
  fv_state* s = const_cast<fv_state*>(cs);
  if (!s || !dst) return fvh::fail(FV_EINVAL, "null argument");
  FV_CUDA_TRY(fvs::enter(s));
  const size_t bytes = (size_t)s->g.member() * s->g.B * sizeof(float);
  FV_CUDA_TRY(cudaMemcpyAsync(dst, s->qA, bytes, kind_from_device(dst_loc), s->stream));
  FV_CUDA_TRY(fvs::leave(s));
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return fvs::check_health(s);
}

extern "C" int fv_set_state(fv_state* s, const float* src, int src_loc) {
  if (!s || !src) return fvh::fail(FV_EINVAL, "null argument");
  FV_CUDA_TRY(fvs::enter(s));
  const size_t bytes = (size_t)s->g.member() * s->g.B * sizeof(float);
  FV_CUDA_TRY(cudaMemcpyAsync(s->qA, src, bytes, kind_to_device(src_loc), s->stream));
  FV_CUDA_TRY(fvs::wavespeed_init(s));
  FV_CUDA_TRY(fvs::leave(s));
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return FV_OK;
}

extern "C" int fv_state_device_ptr(const fv_state* s, float** dptr) {
  if (!s || !dptr) return fvh::fail(FV_EINVAL, "null argument");
  *dptr = s->qA;
  return FV_OK;
}

extern "C" int fv_get_time(const fv_state* cs, double* t, double* next_dt, long long* steps) {
  fv_state* s = const_cast<fv_state*>(cs);
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  std::vector<fvk::Ctrl> c(s->g.B);
  FV_CUDA_TRY(cudaMemcpy(c.data(), s->ctrl, sizeof(fvk::Ctrl) * s->g.B, cudaMemcpyDeviceToHost));
  for (int b = 0; b < s->g.B; ++b) {
    if (t) t[b] = c[b].t;
    if (next_dt) next_dt[b] = c[b].dt;
    if (steps) steps[b] = c[b].step;
  }
  return FV_OK;
}

extern "C" int fv_health(const fv_state* cs, unsigned* flags) {
  fv_state* s = const_cast<fv_state*>(cs);
  if (!s || !flags) return fvh::fail(FV_EINVAL, "null argument");
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  std::vector<fvk::Ctrl> c(s->g.B);
  FV_CUDA_TRY(cudaMemcpy(c.data(), s->ctrl, sizeof(fvk::Ctrl) * s->g.B, cudaMemcpyDeviceToHost));
  for (int b = 0; b < s->g.B; ++b) flags[b] = c[b].health;
  return FV_OK;
}

extern "C" int fv_diagnostics(const fv_state* cs, double* sums) {
  fv_state* s = const_cast<fv_state*>(cs);
  if (!s || !sums) return fvh::fail(FV_EINVAL, "null argument");
  if (s->g.eq == fvk::SPHERE) return fvh::fail(FV_EINVAL, "plain-grid diagnostics do not apply to a sphere state");
  FV_CUDA_TRY(fvs::enter(s));
  FV_CUDA_TRY(fvk::launch_diagnostics(s->g, s->qA, s->diag_partials, s->diag_out, s->stream));
  FV_CUDA_TRY(cudaMemcpyAsync(sums, s->diag_out, sizeof(double) * s->g.B * (s->g.C + 1),
                              cudaMemcpyDeviceToHost, s->stream));
  FV_CUDA_TRY(fvs::leave(s));
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return FV_OK;
}

extern "C" int fv_set_stage_variant(fv_state* s, int variant) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (variant < fvk::STAGE_AUTO || variant > fvk::STAGE_MARCH)
    return fvh::fail(FV_EINVAL, "unknown stage variant");
  if (variant == fvk::STAGE_MARCH && (s->g.nx % 4 != 0 || s->g.nx < 8))
    return fvh::fail(FV_EINVAL, "the row-march kernel needs nx % 4 == 0 and nx >= 8");
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->variant = variant;
  if (s->graph) cudaGraphExecDestroy(s->graph);
  s->graph = nullptr;
  return FV_OK;
}

extern "C" int fv_set_scheme(fv_state* s, int flux, int rk) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (flux < FV_FLUX_HLL || flux > FV_FLUX_HLLC) return fvh::fail(FV_EINVAL, "unknown flux");
  if (rk != 2 && rk != 3) return fvh::fail(FV_EINVAL, "rk must be 2 or 3");
  if (s->g.eq == fvk::SPHERE && (flux == FV_FLUX_LF || rk != 2))
    return fvh::fail(FV_EINVAL, "the sphere step takes HLL, Rusanov, Roe, HLLE or HLLC with SSP-RK2");
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (rk == 3 && !s->qC) {
    const size_t bytes = sizeof(float) * (size_t)s->g.B * (size_t)s->g.member();
    FV_CUDA_TRY(cudaMalloc(&s->qC, bytes));
  }
  s->flux = flux;
  s->rk = rk;
  if (s->graph) cudaGraphExecDestroy(s->graph);
  s->graph = nullptr;
  return FV_OK;
}

extern "C" int fv_set_boundary(fv_state* s, int bc) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (bc != FV_BC_PERIODIC && bc != FV_BC_WALL) return fvh::fail(FV_EINVAL, "unknown boundary condition");
  if (s->g.eq == fvk::SPHERE) return fvh::fail(FV_EINVAL, "a sphere state has no boundary");
  if (bc == FV_BC_WALL && (s->g.nx < 2 || s->g.ny < 2)) return fvh::fail(FV_EINVAL, "walls need nx, ny >= 2");
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->bc = bc;
  if (s->graph) cudaGraphExecDestroy(s->graph);
  s->graph = nullptr;
  return FV_OK;
}

extern "C" int fv_set_bathymetry(fv_state* s, const float* z, int z_loc) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (s->g.eq != fvk::SWE) return fvh::fail(FV_EINVAL, "a bed applies to shallow-water states only");
  if (z && z_loc != FV_HOST && z_loc != FV_DEVICE) return fvh::fail(FV_EINVAL, "z_loc must be FV_HOST or FV_DEVICE");
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (!z) {
    cudaFree(s->zbed);
    s->zbed = nullptr;
  } else {
    const size_t bytes = sizeof(float) * (size_t)s->g.nx * (size_t)s->g.ny;
    if (!s->zbed) FV_CUDA_TRY(cudaMalloc(&s->zbed, bytes));
    FV_CUDA_TRY(cudaMemcpy(s->zbed, z, bytes, z_loc == FV_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice));
  }
  if (s->graph) cudaGraphExecDestroy(s->graph);
  s->graph = nullptr;
  return FV_OK;
}

extern "C" int fv_set_learned_variant(fv_state* s, int variant) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (variant < FV_LEARNED_AUTO || variant > FV_LEARNED_TWO_PASS)
    return fvh::fail(FV_EINVAL, "unknown learned variant");
  if (variant == FV_LEARNED_FUSED && !fvk::learned_fused_supported(s->g.nx, s->g.ny))
    return fvh::fail(FV_EINVAL, "the fused learned kernel needs nx a multiple of 128, at most 1024");
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->learned_variant = variant;
  if (s->graph) cudaGraphExecDestroy(s->graph);
  s->graph = nullptr;
  return FV_OK;
}

extern "C" int fv_set_learned_hmin(fv_state* s, double hmin_frac) {
  if (!s) return fvh::fail(FV_EINVAL, "null state");
  if (!(hmin_frac >= 0.0) || hmin_frac >= 1.0) return fvh::fail(FV_EINVAL, "hmin_frac must be in [0, 1)");
  if (fvs::learned_hmin_fixed(s)) return fvh::fail(FV_EINVAL, "h_min is fixed once the state has taken a learned step");
  s->hmin_frac = (float)hmin_frac;
  return FV_OK;
}

extern "C" int fv_state_stream(const fv_state* s, void** stream) {
  if (!s || !stream) return fvh::fail(FV_EINVAL, "null argument");
  *stream = (void*)s->stream;
  return FV_OK;
}

// ---------------------------------------------------------------------------
// Checkpoints: a host blob holding a header (magic, version, equations,
// batch, grid), every member's control block (time, pending dt, steps,
// health, stop rules) and the state q^n.  Loading it into a state of the same
// shape and equations resumes the run: the following steps are bitwise those
// the saved state would have taken.
// ---------------------------------------------------------------------------
namespace {

struct CkptHeader {
  char magic[8];           // "FVCKPT1\0"
  int eq, C, B, nx, ny;
  int reserved;
  long long ctrl_bytes, state_bytes;
};

constexpr char kCkptMagic[8] = {'F', 'V', 'C', 'K', 'P', 'T', '1', '\0'};

}  // namespace

extern "C" int fv_checkpoint_bytes(const fv_state* s, size_t* bytes) {
  if (!s || !bytes) return fvh::fail(FV_EINVAL, "null argument");
  *bytes = sizeof(CkptHeader) + sizeof(fvk::Ctrl) * (size_t)s->g.B + (size_t)s->g.member() * s->g.B * sizeof(float);
  return FV_OK;
}

extern "C" int fv_checkpoint_save(fv_state* s, void* dst) {
  if (!s || !dst) return fvh::fail(FV_EINVAL, "null argument");
  CkptHeader h{};
  for (int i = 0; i < 8; ++i) h.magic[i] = kCkptMagic[i];
  h.eq = s->g.eq;
  h.C = s->g.C;
  h.B = s->g.B;
  h.nx = s->g.nx;
  h.ny = s->g.ny;
  h.ctrl_bytes = (long long)sizeof(fvk::Ctrl) * s->g.B;
  h.state_bytes = (long long)s->g.member() * s->g.B * (long long)sizeof(float);
  uint8_t* p = static_cast<uint8_t*>(dst);
  memcpy(p, &h, sizeof h);
  FV_CUDA_TRY(fvs::enter(s));
  FV_CUDA_TRY(cudaMemcpyAsync(p + sizeof h, s->ctrl, (size_t)h.ctrl_bytes, cudaMemcpyDeviceToHost, s->stream));
  FV_CUDA_TRY(cudaMemcpyAsync(p + sizeof h + h.ctrl_bytes, s->qA, (size_t)h.state_bytes, cudaMemcpyDeviceToHost,
                              s->stream));
  FV_CUDA_TRY(fvs::leave(s));
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return FV_OK;
}

extern "C" int fv_checkpoint_load(fv_state* s, const void* src) {
  if (!s || !src) return fvh::fail(FV_EINVAL, "null argument");
  CkptHeader h{};
  const uint8_t* p = static_cast<const uint8_t*>(src);
  memcpy(&h, p, sizeof h);
  for (int i = 0; i < 8; ++i)
    if (h.magic[i] != kCkptMagic[i]) return fvh::fail(FV_EINVAL, "not a checkpoint of this library");
  if (h.eq != s->g.eq || h.C != s->g.C || h.B != s->g.B || h.nx != s->g.nx || h.ny != s->g.ny ||
      h.ctrl_bytes != (long long)sizeof(fvk::Ctrl) * s->g.B ||
      h.state_bytes != (long long)s->g.member() * s->g.B * (long long)sizeof(float))
    return fvh::fail(FV_EINVAL, "checkpoint of another equation set, batch or grid");
  FV_CUDA_TRY(fvs::enter(s));
  FV_CUDA_TRY(cudaMemcpyAsync(s->ctrl, p + sizeof h, (size_t)h.ctrl_bytes, cudaMemcpyHostToDevice, s->stream));
  FV_CUDA_TRY(cudaMemcpyAsync(s->qA, p + sizeof h + h.ctrl_bytes, (size_t)h.state_bytes, cudaMemcpyHostToDevice,
                              s->stream));
  FV_CUDA_TRY(fvs::leave(s));
  FV_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return FV_OK;
}
