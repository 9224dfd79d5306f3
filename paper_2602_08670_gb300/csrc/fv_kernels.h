// fv_kernels.h — host-side launchers of the finite-volume kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "fv_common.cuh"

namespace fvk {

// Grid geometry and physical constant of one state.
struct Geom {
  int nx, ny, B, C, eq;   // eq: SWE or EULER
  double dx, dy;
  float phys;             // g (SWE) or gamma (Euler), as used by the FP32 kernels
  double phys_d;          // the same constant in FP64 (diagnostics)
  // Cells [hx, nx - hx) x [hy, ny - hy) are the grid's interior: the CFL
  // reduction, the health bits and the diagnostics cover them only.  A state
  // that is one subdomain of a decomposed grid carries a ring of hx columns
  // and hy rows of its neighbours' cells, refreshed before every stage; a
  // whole periodic grid has hx = hy = 0.
  int hx, hy;
  long long plane() const { return (long long)nx * ny; }
  long long member() const { return plane() * C; }
};

// One SSP-RK2 stage (Eq. 2.19) with MUSCL-minmod faces (Eq. 2.18) and HLL
// fluxes (Eq. 2.15):
//   stage 1: qout = qin + dt L(qin)
//   stage 2: qout = qn/2 + qin/2 + dt L(qin)/2, then the CFL reduction of qout
// qout may alias qn (each cell of qn is read only by the thread writing it).
// variant: STAGE_AUTO (row-march kernel when nx % 4 == 0 and nx >= 8, else
// the shared-memory tile kernel), STAGE_TILE or STAGE_MARCH.  Both kernels
// evaluate the same per-face and per-cell arithmetic, so their results are
// bitwise identical.
enum { STAGE_AUTO = 0, STAGE_TILE = 1, STAGE_MARCH = 2 };
cudaError_t launch_stage_minmod(const Geom& g, int stage, const float* qin, const float* qn,
                                float* qout, Ctrl* ctrl, const DtParams* dp, cudaStream_t s,
                                int variant);

// Boundary on all four sides: periodic, or reflecting walls (mirror ghost
// cells with the momentum normal to the wall negated).
enum { BC_PERIODIC = 0, BC_WALL = 1 };

// Row-march stage with the flux chosen at run time (fvk::Flux) and stage
// kind 1 (q1 = q^n + dt L), 2 (Heun), 3, 4 (SSP-RK3 stages 2 and 3; the
// CFL reduction in 2 and 4); `bc` BC_*, `z` the shallow-water bed [ny][nx]
// on the device (bed-slope source of Eq. 2.3) or null.  Needs
// march_supported(g) (and ny >= 2 with walls).
bool march_supported(const Geom& g);
cudaError_t launch_stage_general(const Geom& g, int stage, int flux, const float* qin, const float* qn,
                                 float* qout, Ctrl* ctrl, const DtParams* dp, cudaStream_t s,
                                 int bc = BC_PERIODIC, const float* z = nullptr);

// Shallow water on the sphere (fv_sphere.cu): metric planes of the nx x ny
// two-hemisphere grid (computed once per state), the Courant-rate reduction
// of a state, and one SSP-RK2 step (q^n in qa, updated in place; stage in qb).
long long sphere_metric_floats(int nx, int ny);
long long sphere_centre_offset(int nx, int ny);   // [3][ny][nx] unit cell centres
long long sphere_area_offset(int nx, int ny);     // [ny][nx] spherical cell areas
cudaError_t launch_sphere_metrics(float* M, int nx, int ny, cudaStream_t s);
cudaError_t launch_sphere_wavespeed(const Geom& g, const float* q, const float* M, Ctrl* ctrl,
                                    const DtParams* dp, cudaStream_t s);
cudaError_t enqueue_sphere_step(const Geom& g, int flux, float* qa, float* qb, const float* M, float omega,
                                Ctrl* ctrl, const DtParams* dp, cudaStream_t s);

// Wave-speed reduction of q that sets each member's dt without advancing
// time (state creation, fv_set_state); member >= 0: that member only.
cudaError_t launch_wavespeed_init(const Geom& g, const float* q, Ctrl* ctrl, const DtParams* dp,
                                  cudaStream_t s, int member = -1);

// FP64 sums [B][C+1] into device memory `out` (deterministic order).
// `partials` must hold diag_partials_size(g) doubles.
long long diag_partials_size(const Geom& g);
cudaError_t launch_diagnostics(const Geom& g, const float* q, double* partials, double* out,
                               cudaStream_t s);

// Set t_end on every member, clamp the pending dt to it and set `done`.
cudaError_t launch_set_t_end(Ctrl* ctrl, int B, double t_end, cudaStream_t s);

}  // namespace fvk
