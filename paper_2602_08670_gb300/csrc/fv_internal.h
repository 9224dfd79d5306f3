// fv_internal.h — the state object behind the opaque fv_state handle and the
// internal functions shared by the API translation units.
#pragma once

#include <cuda_runtime.h>

#include "fv_common.cuh"
#include "fv_kernels.h"

namespace snk {
struct Net;
}

namespace fvk {
// Learned stage as one persistent kernel (CNN + learned faces + HLL + RK),
// for nx a multiple of 128 up to 1024.
bool learned_fused_supported(int nx, int ny);
cudaError_t launch_learned_fused(const Geom& g, int stage, const float* qin, const float* qn,
                                 float* qout, const snk::Net& net, const float* hmin, Ctrl* ctrl,
                                 const DtParams* dp, cudaStream_t s);
// One plain step with flux `flux` (fvk::Flux) and integrator `rk` (2: SSP-RK2,
// 3: SSP-RK3); q^n in qa (updated in place), stages in qb and qc.  `variant`
// as for the HLL stages (STAGE_TILE forces the tile kernel); `bc` FV_BC_*,
// `z` the shallow-water bed [ny][nx] on the device or null.
cudaError_t enqueue_scheme_step(const Geom& g, int flux, int rk, float* qa, float* qb, float* qc,
                                Ctrl* ctrl, const DtParams* dp, cudaStream_t s, int variant, int bc,
                                const float* z);
cudaError_t launch_stage_learned(const Geom& g, int stage, const float* qin, const float* qn,
                                 float* qout, const float* w, const float* hmin, Ctrl* ctrl,
                                 const DtParams* dp, cudaStream_t s);
// One SSP-RK2 stage of the face-state path (Section 2.5.3, third approach)
// from the side states [B][12][plane] of qin.
cudaError_t launch_stage_face(const Geom& g, int stage, const float* qin, const float* qn, float* qout,
                              const float* sides, Ctrl* ctrl, const DtParams* dp, cudaStream_t s);
}

struct fv_learned_ws;   // per-state workspace of the learned step (fv_learned.cu)

struct fv_state {
  fvk::Geom g{};
  double lx = 1.0, ly = 1.0;
  int dt_mode = FV_DT_ADAPTIVE;
  cudaStream_t stream = nullptr;       // all work of the state runs here
  cudaStream_t user_stream = nullptr;  // caller's stream, or null
  bool own_stream = false;             // stream created by the library
  cudaEvent_t ev = nullptr;
  float* qA = nullptr;                 // q^n, and q^{n+1} after stage 2
  float* qB = nullptr;                 // q^(1), the stage-1 output
  fvk::Ctrl* ctrl = nullptr;           // device [B]
  fvk::DtParams* dp = nullptr;         // device
  fvk::DtParams dp_host{};
  double* replay = nullptr;            // device REPLAY dt sequence
  double* diag_partials = nullptr;
  double* diag_out = nullptr;
  cudaGraphExec_t graph = nullptr;     // captured chunk of steps
  long graph_steps = 0;
  const fv_net* graph_net = nullptr;
  fv_learned_ws* lws = nullptr;        // learned-step workspace (lazily created)
  float hmin_frac = 1e-3f;             // learned faces: h_min = hmin_frac * mean depth
  int variant = 0;                     // stage kernel choice (fvk::STAGE_*)
  int learned_variant = 0;             // FV_LEARNED_AUTO / _FUSED / _TWO_PASS
  int flux = 0;                        // FV_FLUX_* of the plain step
  int rk = 2;                          // 2: SSP-RK2, 3: SSP-RK3
  float* qC = nullptr;                 // q^(2) of SSP-RK3 (allocated on first use)
  int bc = 0;                          // FV_BC_PERIODIC or FV_BC_WALL
  float* zbed = nullptr;               // shallow-water bed [ny][nx] (device), or null
  float* sphere = nullptr;             // sphere grid metrics (device), SPHERE states only
  float omega = 0.f;                   // rotation rate of the sphere (Coriolis)
};

namespace fvs {
int state_alloc(fv_state* s);
cudaError_t enqueue_plain_stage(fv_state* s, int stage);   // HLL, SSP-RK2, periodic, flat bed
void state_free(fv_state* s);
cudaError_t enter(fv_state* s);
cudaError_t leave(fv_state* s);
cudaError_t enqueue_plain_step(fv_state* s);
cudaError_t enqueue_step(fv_state* s, const fv_net* net);
int check_health(fv_state* s);
cudaError_t wavespeed_init(fv_state* s);                // dt of the current state (no time advance)
// learned path (fv_learned.cu)
int learned_prepare(fv_state* s, const fv_net* net);  // host side, before enqueueing
cudaError_t enqueue_learned_step(fv_state* s, const fv_net* net);
cudaError_t enqueue_learned_stage(fv_state* s, const fv_net* net, int stage);   // 1 or 2
int learned_set_hmin_values(fv_state* s, const double* hmin);   // absolute h_min per member
void learned_workspace_free(fv_state* s);
bool learned_hmin_fixed(const fv_state* s);           // a stencil-network step has set h_min
float* learned_hmin_ptr(fv_state* s);                 // device [B] h_min, or null
long long learned_ws_bytes(const fv_state* s);        // device memory of the learned workspace
long long state_device_bytes(const fv_state* s);      // device memory held by the state
int net_check(const fv_net* n);                      // device error word of a network
}  // namespace fvs
