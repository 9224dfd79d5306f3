/*
 * fv.h — C ABI of the GB300 finite-volume library (libfv.so).
 *
 * Explicit finite-volume time stepping of the 2D shallow-water equations
 * (Eq. 2.3, flat bed) and the 2D Euler equations (Section 4.2, ideal gas,
 * Eq. 2.4) on periodic Cartesian grids: MUSCL reconstruction with the MINMOD
 * limiter (Eq. 2.18), the HLL numerical flux (Eq. 2.15) in the face-normal
 * frame (Eq. 2.24), the conservative update (Eqs. 2.9, 2.23) and Heun /
 * SSP-RK2 time integration (Eq. 2.19) with the CFL rule (Eq. 2.10).  The
 * learned variant (Section 2.5.3, fourth approach) replaces MINMOD by
 * CNN-predicted, sum-to-one stencil coefficients.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an int status: FV_OK (0), FV_PENDING (1), or a
 *    negative fv_status error.  fv_last_error() gives a thread-local message
 *    for the last failing call of the calling thread.
 *  - State layout: q[B][C][ny][nx], FP32, x fastest, contiguous.  SWE: C = 3,
 *    (h, hu, hv).  Euler: C = 4, (rho, rho u, rho v, E).
 *  - Pointer location tags: FV_HOST (pageable or pinned host memory) or
 *    FV_DEVICE (device memory of the current CUDA device).  Caller buffers are
 *    borrowed for the duration of the call only.
 *  - Handles (fv_state, fv_net, fv_server) are opaque; the library owns every
 *    device allocation it makes and frees it in the matching fv_destroy_*.
 *  - stream: a cudaStream_t passed as void* (e.g. PyTorch's current stream).
 *    A created (non-default) stream is used directly: every kernel of the
 *    handle runs on it.  NULL, cudaStreamLegacy or cudaStreamPerThread make
 *    the library create its own stream for the handle, ordered after work
 *    already queued on the given default stream at each call, and before work
 *    queued there afterwards.  Calls that return host data synchronise.
 *  - Device-side failures (NaN/Inf, h <= 0, rho <= 0, p <= 0, Courant number
 *    above 1 in FIXED/REPLAY mode) are recorded in a per-member health word and
 *    reported as FV_EUNSTABLE by the next synchronising call.
 */
#ifndef FV_H_
#define FV_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FV_OK = 0,
  FV_PENDING = 1,      /* poll(): the request is not finished yet            */
  FV_EINVAL = -1,      /* bad argument (null pointer, size, mode, ...)       */
  FV_ENOMEM = -2,      /* a device or host allocation failed                  */
  FV_EUNSTABLE = -3,   /* health word set on the device (see above)           */
  FV_ETIMEOUT = -4,    /* a bounded wait gave up                              */
  FV_EBUSY = -5,       /* submit(): the request can never fit the budget      */
  FV_ECUDA = -6,       /* a CUDA runtime call failed                          */
  FV_ENOTFOUND = -7    /* unknown ticket                                      */
} fv_status;

enum { FV_HOST = 0, FV_DEVICE = 1 };
enum { FV_EQ_SWE = 0, FV_EQ_EULER = 1 };
enum { FV_DT_ADAPTIVE = 0, FV_DT_FIXED = 1, FV_DT_REPLAY = 2 };

/* Health bits (fv_health). */
enum {
  FV_HEALTH_NONFINITE = 1u,   /* NaN or Inf in a stage output               */
  FV_HEALTH_NONPOSITIVE = 2u, /* h <= 0 (SWE), rho <= 0 or p <= 0 (Euler)    */
  FV_HEALTH_CFL = 4u,         /* Courant number > 1 with a FIXED/REPLAY dt   */
  FV_HEALTH_REPLAY_END = 8u   /* REPLAY ran past the supplied dt sequence    */
};

/* Periodic grid [0, lx) x [0, ly) with nx x ny cells of size lx/nx x ly/ny
 * (Section 2.3.1: N cells per direction, centres (i + 1/2) dx),
 * and `batch` independent members that share the grid. */
typedef struct { int nx, ny, batch; double lx, ly; } fv_grid;

/* Time-step control (Eq. 2.10 with the Courant number of the unsplit 2D
 * update, C = dt * max_cells((|u| + c)/dx + (|v| + c)/dy)).  ADAPTIVE:
 * dt = cfl / max_cells((|u| + c)/dx + (|v| + c)/dy), per member, evaluated
 * on q^n.  FIXED: dt = dt_fixed.  REPLAY: step n uses the n-th value given to
 * fv_set_replay_dt() for every member.  FIXED and REPLAY raise
 * FV_HEALTH_CFL when C exceeds 1. */
typedef struct { double g; double cfl; int dt_mode; double dt_fixed; } fv_swe_params;
typedef struct { double gamma; double cfl; int dt_mode; double dt_fixed; } fv_euler_params;
/* Shallow water on the rotating unit sphere: gravity g and rotation rate
 * omega in the units of the state (e.g. Earth radii and days). */
typedef struct { double g; double omega; double cfl; int dt_mode; double dt_fixed; } fv_sphere_params;

typedef struct fv_state fv_state;
typedef struct fv_net fv_net;
typedef struct fv_server fv_server;

/* Thread-local message of the last failing call ("" if none). */
const char* fv_last_error(void);

/* ---------------------------------------------------------------------------
 * States
 * ------------------------------------------------------------------------- */

/* Create a shallow-water state (Eq. 2.3, S = 0).  q0: [batch][3][ny][nx] FP32
 * at location q0_loc; copied into library-owned device memory.  The initial
 * dt is computed on the device.  Requires nx, ny >= 1, batch >= 1, g > 0,
 * h > 0 everywhere (else FV_EUNSTABLE at the first synchronising call).
 * Errors: FV_EINVAL, FV_ENOMEM, FV_ECUDA. */
int swe_init(const fv_grid* grid, const fv_swe_params* params, const float* q0,
             int q0_loc, void* stream, fv_state** out);

/* Create a 2D Euler state (Section 4.2, ideal gas Eq. 2.4 with gamma > 1).
 * q0: [batch][4][ny][nx] conserved variables (rho, rho u, rho v, E). */
int euler_init(const fv_grid* grid, const fv_euler_params* params, const float* q0,
               int q0_loc, void* stream, fv_state** out);

/* Free a state and everything it owns (NULL is accepted). */
/* Shallow water on the unit sphere (Sections 2.4 and 4.3).  q0: [batch][4]
 * [ny][nx] FP32, (h, hu, hv, hw) with a Cartesian momentum, on the
 * logically rectangular grid of two hemispheres: nx = 2 ny cells on the
 * computational rectangle [-3, 1] x [-1, 1], the right square the upper
 * hemisphere (the disk mapping D(d) = d / sqrt 2, R(d) = 1 lifted by
 * z = sqrt(1 - x^2 - y^2), Eq. 2.25), the left square the lower one; x is
 * periodic and the cell above row ny - 1 of column i is row ny - 1 of column
 * nx - 1 - i.  The step: MUSCL-minmod faces in the logical directions, the
 * HLL flux in each edge's (normal, tangent, radial) frame with great-circle
 * edge lengths and spherical cell areas, Eq. 3.1's correction on the
 * momenta, Coriolis (Eq. 3.2), projection of the momentum onto the tangent
 * plane after each stage, SSP-RK2, dt from the Courant rate
 * (|m| / h + sqrt(g h)) * perimeter / (2 area).  The grid metrics are
 * computed once on the device (FP64, stored FP32) and shared by the members.
 * fv_step / fv_rollout / fv_get_state / fv_set_state / fv_get_time /
 * fv_health apply; fv_set_scheme accepts HLL, Rusanov, Roe, HLLE or HLLC
 * with SSP-RK2 (the tangential momenta m.t and m.r passive; Lax-Friedrichs
 * and SSP-RK3 are FV_EINVAL), and
 * fv_set_boundary, fv_set_bathymetry, fv_diagnostics and learned steps
 * return FV_EINVAL.  Errors: FV_EINVAL (nx != 2 ny, ny < 2, g <= 0),
 * FV_ENOMEM, FV_ECUDA. */
int sphere_init(int nx, int ny, int batch, const fv_sphere_params* p, const float* q0, int q0_loc,
                void* stream, fv_state** out);

/* The grid of a sphere state: unit cell centres [3][ny][nx] (x, y, z
 * planes) and spherical cell areas [ny][nx], FP32, into host or device
 * memory per loc (either pointer may be NULL).  FV_EINVAL for another
 * state. */
int sphere_get_cells(const fv_state* s, float* centres, float* areas, int loc);

int fv_destroy_state(fv_state* s);

/* REPLAY mode: the dt of step k (k = 0..n-1, counted from the state's
 * creation) for every member.  dts is a host array of n doubles, copied. */
int fv_set_replay_dt(fv_state* s, const double* dts, long n);

/* Enqueue one SSP-RK2 step (Eq. 2.19) of every member on the state's
 * stream; asynchronous.  net == NULL: MUSCL-minmod reconstruction.  net !=
 * NULL (SWE only): learned reconstruction with minmod fallback. */
int fv_step(fv_state* s, const fv_net* net);

/* Enqueue up to nsteps steps as replays of a captured CUDA graph and wait
 * for them.  t_end > 0 stops every member at simulated time t_end exactly
 * (its last step shortened, later steps skipped on the device); t_end <= 0
 * ignores it.  If snaps != NULL and snap_every > 0, the state after every
 * snap_every-th step is written to snaps (location snaps_loc) as
 * [nsteps/snap_every][batch][C][ny][nx].  t_out (host, [batch], may be NULL)
 * receives each member's simulated time.  Returns FV_EUNSTABLE if a health
 * bit was raised. */
int fv_rollout(fv_state* s, const fv_net* net, long nsteps, double t_end,
               float* snaps, int snaps_loc, int snap_every, double* t_out);

/* Enqueue nsteps steps (graph replays of 32-step chunks plus a direct tail)
 * and return without waiting; the state's t_end setting is left as it is.
 * Health is reported by the next synchronising call. */
int fv_enqueue_steps(fv_state* s, const fv_net* net, long nsteps);

/* Wait for the state's stream and report health (FV_OK or FV_EUNSTABLE). */
int fv_sync(fv_state* s);

/* Copy the current state to dst ([batch][C][ny][nx], location dst_loc). */
int fv_get_state(const fv_state* s, float* dst, int dst_loc);

/* Overwrite the current state from src (same shape); time and step count are
 * kept, the dt of the next step is recomputed (ADAPTIVE). */
int fv_set_state(fv_state* s, const float* src, int src_loc);

/* Device pointer of the state buffer (owned by the state; valid until the
 * next fv_destroy_state).  For zero-copy binding layers. */
int fv_state_device_ptr(const fv_state* s, float** dptr);

/* Stage-kernel implementation of the plain step (every flux and integrator
 * of fv_set_scheme): 0 = automatic (row-march kernel when nx is a multiple of
 * 4 and >= 8, else the shared-memory tile kernel), 1 = tile kernel, 2 =
 * row-march kernel (FV_EINVAL if nx does not allow it).  Both evaluate the same formulas per face and per cell; the
 * approximate reciprocal and square root may be scheduled differently, so
 * results agree to a few ulps, not bitwise.  The choice only changes speed. */
int fv_set_stage_variant(fv_state* s, int variant);

/* Numerical flux and time integrator of the plain step (Section 2.3.3):
 *  flux: FV_FLUX_HLL (Eq. 2.15, default), FV_FLUX_RUSANOV (Eq. 2.12),
 *        FV_FLUX_LF (Lax-Friedrichs, Eq. 2.11, with viscosity dx/(4 dt) on x
 *        faces and dy/(4 dt) on y faces: the paper's one-dimensional dx/(2 dt)
 *        in both directions of the unsplit update amplifies the grid-scale
 *        checkerboard by -3 for every dt), FV_FLUX_ROE (Eqs. 2.13-2.14, Roe
 *        averages, no entropy fix), FV_FLUX_HLLE (Eq. 2.16, speeds clamped by
 *        the Roe state's and by 0), FV_FLUX_HLLC (Eq. 2.17, HLL outer speeds,
 *        middle speed from the jump conditions);
 *  rk:   2 = Heun / SSP-RK2 (Eq. 2.19, default), 3 = SSP-RK3 (Eq. 2.20,
 *        printed as fourth order; it is the three-stage third-order scheme).
 * Reconstruction (MUSCL-minmod), rotation, divergence and the CFL rule are
 * unchanged.  The HLL / SSP-RK2 pair runs the row-march kernels; the others
 * a shared-memory tile kernel with the flux chosen per launch.  rk = 3
 * allocates one more state buffer on first use.  The learned step requires
 * HLL and SSP-RK2 (FV_EINVAL otherwise).  Synchronises the state's stream. */
enum { FV_FLUX_HLL = 0, FV_FLUX_RUSANOV = 1, FV_FLUX_LF = 2, FV_FLUX_ROE = 3, FV_FLUX_HLLE = 4,
       FV_FLUX_HLLC = 5 };
int fv_set_scheme(fv_state* s, int flux, int rk);

/* Boundary condition on all four sides (shallow water and Euler):
 * FV_BC_PERIODIC (default) or FV_BC_WALL, a reflecting wall as in the
 * bathymetry test of Section 4.2: the halo cells mirror the interior with the
 * momentum normal to the wall negated, so no mass crosses it.  Walls run in
 * the plain step's stage kernels (row march or tile, per
 * fv_set_stage_variant; any flux and integrator of fv_set_scheme); the
 * learned step stays periodic (FV_EINVAL there).  FV_EINVAL for an unknown
 * value or a grid narrower than 2 cells. */
enum { FV_BC_PERIODIC = 0, FV_BC_WALL = 1 };
int fv_set_boundary(fv_state* s, int bc);

/* Bed z of a shallow-water state (Eq. 2.3): the momentum equations gain
 * -g h dz/dx and -g h dz/dy, with z given at the cell centres as FP32
 * [ny][nx] (one bed for every member; host or device memory per z_loc,
 * copied, not retained) and its slope taken as the centred difference
 * (z_{i+1} - z_{i-1}) / (2 dx) (mirrored at walls, wrapped when periodic).
 * z = NULL returns to the flat bed.  Runs in the plain step's stage kernels;
 * the learned step needs a flat bed.  FV_EINVAL for an Euler state or a bad
 * z_loc. */
int fv_set_bathymetry(fv_state* s, const float* z, int z_loc);

/* Implementation of the learned step (Section 2.5.3, fourth approach):
 *  FV_LEARNED_AUTO (0): the fused kernel where the grid allows it, else the
 *    two-pass path;
 *  FV_LEARNED_FUSED (1): one persistent kernel per Runge-Kutta stage that
 *    evaluates the CNN row by row on the tensor cores and uses the
 *    coefficients straight from on-chip memory (nx a multiple of 128, at most
 *    1024; FV_EINVAL otherwise);
 *  FV_LEARNED_TWO_PASS (2): the CNN writes the coefficients of every cell to
 *    device memory, then a stage kernel reads them (nx in {8, 16, 32, 64} or
 *    a multiple of 128).
 * Both use BF16 operands with FP32 accumulation and the same per-face
 * arithmetic; the first layer sums its taps in a different order, so results
 * agree to rounding, not bitwise. */
enum { FV_LEARNED_AUTO = 0, FV_LEARNED_FUSED = 1, FV_LEARNED_TWO_PASS = 2 };
int fv_set_learned_variant(fv_state* s, int variant);

/* The CUDA stream (cudaStream_t as void*) on which the state's kernels run,
 * owned by the state; for callers that time or order work against it. */
int fv_state_stream(const fv_state* s, void** stream);

/* Per member: simulated time t (host [batch]), the dt the next step will use
 * (host [batch]) and the number of completed steps (host [batch]); any
 * pointer may be NULL. */
int fv_get_time(const fv_state* s, double* t, double* next_dt, long long* steps);

/* Per member health bits (host [batch]). */
int fv_health(const fv_state* s, unsigned* flags);

/* FP64 global sums per member, host [batch][C+1]: the integral of each
 * conserved variable (sum of cell values times dx dy), then SWE: total energy
 * of Eq. 5.1, integral of g h^2/2 + (u^2+v^2) h/2; Euler: kinetic energy,
 * integral of rho (u^2+v^2)/2.  Deterministic (fixed reduction order). */
int fv_diagnostics(const fv_state* s, double* sums);

/* Learned step: the positivity threshold h_min = hmin_frac * (mean depth of
 * each member when its first learned step is taken; the mean depth is
 * conserved).  Learned face states with a depth below h_min fall back to the
 * MUSCL-minmod states.  Default 1e-3.  Must be set before the first learned
 * step (FV_EINVAL after). */
int fv_set_learned_hmin(fv_state* s, double hmin_frac);

/* The sums of fv_diagnostics() for a state the caller holds (q: device
 * [batch][C][ny][nx], C = 3 for FV_EQ_SWE with phys = g, 4 for FV_EQ_EULER
 * with phys = gamma, periodic lx x ly domain), computed without allocating
 * any device or host memory.  The paper has no counterpart: this entry point
 * serves callers that cannot allocate once running (a fixed device-memory
 * budget handed out up front, allocation-free real-time loops or host
 * callbacks, frameworks that own all device memory through their own pool).
 * The reduction scratch is a fixed array of 320 slots in the library that
 * every GPU loading it keeps until the process exits: batch * (C + 1) must
 * be at most 320 (80 shallow-water or 64 Euler members), else FV_EINVAL.
 * sums: [batch][C+1] at sums_loc; FV_HOST returns after the result is
 * copied, FV_DEVICE only enqueues on `stream` (cudaStream_t, NULL = default
 * stream).  The first call on a device looks up the scratch address with
 * that device current; make it before any stream capture.  That first call
 * may also be the one that loads the library's device code on the device
 * (CUDA loads modules lazily by default), which is when the fixed scratch is
 * reserved: a caller whose running phase must not allocate makes one warm-up
 * call before entering it.  All calls share
 * the scratch, so calls that overlap on the GPU (other streams, other host
 * threads) race; every slot a call reads is written by that call first. */
int fv_diagnostics_noalloc(const float* q, int eq, int batch, int ny, int nx, double lx, double ly,
                           double phys, double* sums, int sums_loc, void* stream);

/* Checkpoints.  fv_checkpoint_bytes gives the size of the host blob that
 * fv_checkpoint_save fills (synchronous): a header (equations, batch, grid),
 * every member's control block (time, pending dt, completed steps, health,
 * stop rules) and the state q^n.  fv_checkpoint_load restores such a blob
 * into a state of the same equations, batch and grid (FV_EINVAL otherwise);
 * the steps that follow are bitwise those the saved state would have taken.
 * Scheme settings (flux, boundary, bed, replay sequence, network) belong to
 * the state object, not to the checkpoint. */
int fv_checkpoint_bytes(const fv_state* s, size_t* bytes);
int fv_checkpoint_save(fv_state* s, void* dst);
int fv_checkpoint_load(fv_state* s, const void* src);

/* ---------------------------------------------------------------------------
 * Subdomains of a block-decomposed grid
 *
 * The explicit step (Eqs. 2.9, 2.18, 2.19, 2.23) reads a bounded stencil, so
 * a grid splits into px x py blocks that each advance on their own once a
 * ring of their neighbours' cells is in place.  A subdomain is an ordinary
 * state of (nx/px + 2 hx) x (ny/py + 2 hy) cells: its interior plus a ring of
 * hx columns and hy rows copied from the periodic neighbours before every
 * Runge-Kutta stage (hx, hy = 2 for the plain MUSCL-minmod step; 6 rows for
 * the learned step, whose CNN adds 4 cells of reach to the 2 of the
 * reconstruction, rounded up to keep rows 16-byte aligned).  The stage
 * kernels also compute the ring cells (with wrong neighbours); the next
 * refresh overwrites them.  One step of a decomposed grid is
 *   fv_halo_exchange(buf 0); fv_enqueue_stage(1) on every subdomain;
 *   fv_halo_exchange(buf 1); fv_enqueue_stage(2) on every subdomain;
 *   fv_reduce_dt
 * and its interiors equal the undecomposed grid's cells bitwise (the
 * per-cell arithmetic does not depend on the cell's place in the grid, and
 * the next dt is the minimum over the subdomains).  Between processes the
 * ring travels as packed strips (fv_halo_pack / fv_halo_unpack; x first,
 * then y over the full width, which carries the corners) and the dt as a
 * minimum over processes (fv_get_time / fv_set_dt).
 * ------------------------------------------------------------------------- */

/* Declare the outer hx columns and hy rows of s a ring: the CFL reduction,
 * the health bits and fv_diagnostics cover the interior [hx, nx-hx) x
 * [hy, ny-hy) only, and the pending dt is recomputed from the interior.
 * Needs 4 hx <= nx, 4 hy <= ny, a periodic flat-bed planar state.  The fused
 * learned kernel takes rings of rows only (hx = 0).  Synchronous;
 * FV_EUNSTABLE if the interior is not a physical state. */
int fv_set_halo(fv_state* s, int hx, int hy);

/* Enqueue one SSP-RK2 stage (Eq. 2.19): stage 1 maps q^n to the stage state,
 * stage 2 combines them into q^{n+1} and closes the step (time, next dt).
 * net = NULL: the plain HLL/MUSCL-minmod stage; else the learned stage of a
 * stencil or face-state network.  Asynchronous on the state's stream;
 * FV_EINVAL for other schemes, walls or a bed. */
int fv_enqueue_stage(fv_state* s, const fv_net* net, int stage);

/* Fill the ring of buffer `buf` (0: q^n, the input of stage 1; 1: the stage
 * state, the input of stage 2) of px * py subdomains of one process,
 * subs[iy * px + ix] holding block (ix, iy) of the periodic grid, from the
 * interiors of the blocks that own those cells.  All subdomains: same
 * equations, batch, shape and ring; at most 64.  One kernel on subs[0]'s
 * stream, ordered after and before the other subdomains' streams.  A split
 * direction needs a ring (FV_EINVAL). */
int fv_halo_exchange(fv_state* const* subs, int px, int py, int buf);

/* Set every member's pending dt of the n subdomains to its minimum over them
 * (after stage 2, before the next step).  Asynchronous, ordered like
 * fv_halo_exchange. */
int fv_reduce_dt(fv_state* const* subs, int n);

/* Copy the interior strip next to side `side` (0 west, 1 east, 2 south,
 * 3 north) of buffer `buf` into dst (device, fv_halo_strip_floats floats,
 * [B][C][rows][cols]), or write src into that side's ring.  West/east strips
 * span the interior rows, south/north strips the full width: exchange west
 * and east first, then south and north.  Asynchronous on the state's
 * stream. */
int fv_halo_pack(fv_state* s, int buf, int side, float* dst);
int fv_halo_unpack(fv_state* s, int buf, int side, const float* src);
int fv_halo_strip_floats(const fv_state* s, int side, long long* n);

/* Set every member's pending dt (host [B], >= 0; e.g. the minimum over the
 * processes of a decomposed grid).  Synchronous. */
int fv_set_dt(fv_state* s, const double* dt);

/* Positivity threshold of the learned faces as absolute depths per member
 * (host [B]) instead of a fraction of the state's own mean depth: the
 * subdomains of one grid share the whole grid's threshold.  Before the first
 * learned step (FV_EINVAL after). */
int fv_set_learned_hmin_values(fv_state* s, const double* hmin);

/* ---------------------------------------------------------------------------
 * Learned stencil network (Section 2.5.3, fourth approach)
 *
 * x = (q - mean) / std per channel; four 3x3 convolutions with periodic
 * padding, 3 -> 32 -> 32 -> 32 -> 36 channels, ReLU after the first three;
 * BF16 operands, FP32 accumulation on the tensor cores.  The 36 outputs of
 * cell i are r[((dir * 3 + var) * 2 + side) * 3 + tap] (dir 0 = x, 1 = y;
 * side 0 = Q^L of face i+1/2 on cells {i-1, i, i+1}, side 1 = Q^R on
 * {i, i+1, i+2}); each 3-tap stencil is normalised to w = e_centre + r -
 * mean(r), so the weights sum to one and r = 0 gives the first-order scheme.
 * ------------------------------------------------------------------------- */

/* Number of parameters: W1[32][3][3][3] b1[32] W2[32][32][3][3] b2[32]
 * W3[32][32][3][3] b3[32] W4[36][32][3][3] b4[36], concatenated in that
 * order (PyTorch Conv2d layout). */
#define FV_NET_PARAMS 29796

/* Create a network.  params: host [FV_NET_PARAMS] FP32 (NULL = all zeros:
 * the first-order scheme); norm: host [6] = mean[3], std[3] of (h, hu, hv)
 * (NULL = 0 and 1).  Errors: FV_EINVAL, FV_ENOMEM, FV_ECUDA. */
int stencil_net_create(const float* params, const float* norm, fv_net** out);
int stencil_net_destroy(fv_net* n);

/* Replace / read the FP32 parameters ([fv_net_num_params(n)]: FV_NET_PARAMS
 * or, for a face-state network, FV_FACE_NET_PARAMS; location loc). */
int stencil_net_set_params(fv_net* n, const float* params, int loc);
int stencil_net_get_params(const fv_net* n, float* params, int loc);

/* Forward on q (device [B][3][ny][nx] FP32): coeffs (device [B][36][ny][nx]
 * FP32) receives the normalised stencil weights, or the raw network outputs
 * r if raw != 0.  nx must be 8, 16, 32, 64 or a multiple of 128 and nx*ny a
 * multiple of 128 (FV_EINVAL otherwise).  stream: cudaStream_t or NULL (the
 * network's own stream); the call waits for completion.  FV_ETIMEOUT if a
 * bounded tensor-core wait gave up. */
int stencil_net_forward(const fv_net* n, const float* q, int B, int ny, int nx, float* coeffs,
                        int raw, void* stream);

/* stencil_net_forward / _backward and face_net_forward / _backward use a
 * workspace held by the network: calls on one network from several threads
 * must be serialised by the caller.  Steps (fv_step, fv_rollout, the server)
 * only read a network's parameters and keep their workspaces in the state.
 *
 * Vector-Jacobian product of stencil_net_forward at q (the forward is
 * recomputed): dcoeffs (device [B][36][ny][nx] FP32) is the cotangent of the
 * normalised coefficients; the parameter gradient is ADDED to dparams
 * (device [FV_NET_PARAMS]) and, if dq != NULL, the cotangent of q is ADDED
 * to dq (device [B][3][ny][nx]).  Cotangents between layers are BF16
 * (tensor-core operands), weight gradients FP32 with a deterministic
 * reduction.  Grid rules, stream and errors as stencil_net_forward. */
int stencil_net_backward(fv_net* n, const float* q, int B, int ny, int nx, const float* dcoeffs,
                         float* dq, float* dparams, void* stream);

/* ---------------------------------------------------------------------------
 * Face-state network (Section 2.5.3, third approach; Section 5.3)
 *
 * A CNN gives each cell the states on its four sides directly.  Architecture:
 * x = (q - mean) / std; four 3x3 periodic convolutions 3 -> 32 -> 32 -> 32
 * -> 12 with GeLU (x Phi(x), erf form) after the first three; BF16 operands,
 * FP32 accumulation on the tensor cores.  Output channel 3 s + v is side s
 * (0 west, 1 east, 2 south, 3 north) of variable v (h, hu, hv); depths are
 * Softplus(r), momenta mean_v + std_v r.  The flux through the face between
 * cells i-1 and i is HLL of (east state of i-1, west state of i); in y of
 * (north state of j-1, south state of j).  fv_step, fv_enqueue_steps,
 * fv_rollout and the server take a face-state network wherever they take a
 * stencil network (HLL, SSP-RK2, periodic flat bed, adaptive or fixed dt;
 * the network runs at both stages).  stencil_net_destroy, _set_params,
 * _get_params and _adam_step accept either kind, with fv_net_num_params()
 * parameters, and so do the training tapes (fv_tape_*: dparams then holds
 * FV_FACE_NET_PARAMS floats; the tape keeps the BF16 pre-activations for
 * the GeLU derivative).
 * ------------------------------------------------------------------------- */

/* W1[32][3][3][3] b1[32] W2[32][32][3][3] b2[32] W3[32][32][3][3] b3[32]
 * W4[12][32][3][3] b4[12] (PyTorch Conv2d layout). */
#define FV_FACE_NET_PARAMS 22860

/* Create a face-state network; params host [FV_FACE_NET_PARAMS] FP32 (NULL =
 * all zeros), norm as for stencil_net_create.  Errors: FV_EINVAL, FV_ENOMEM,
 * FV_ECUDA. */
int face_net_create(const float* params, const float* norm, fv_net** out);

/* Forward on q (device [B][3][ny][nx] FP32): sides (device [B][12][ny][nx]
 * FP32) receives the side states, or the raw network outputs r if raw != 0.
 * Grid rules, stream and errors as stencil_net_forward; FV_EINVAL for a
 * stencil network. */
int face_net_forward(const fv_net* n, const float* q, int B, int ny, int nx, float* sides, int raw,
                     void* stream);

/* Vector-Jacobian product of face_net_forward at q: dsides (device
 * [B][12][ny][nx]) is the cotangent of the side states; the gradient is
 * ADDED to dparams (device [FV_FACE_NET_PARAMS]) and, if dq != NULL, to dq.
 * As stencil_net_backward otherwise. */
int face_net_backward(fv_net* n, const float* q, int B, int ny, int nx, const float* dsides, float* dq,
                      float* dparams, void* stream);

/* Kind of a network: 0 = stencil (fourth approach), 1 = face-state (third);
 * -1 for NULL.  Parameter count of its kind (0 for NULL). */
int fv_net_kind(const fv_net* n);
int fv_net_num_params(const fv_net* n);

/* Coarse graining (Section 2.5.1): coarse[p][j][i] = mean of the factor x
 * factor block of fine[p][.][.] (FP64 sum), for `planes` planes of ny x nx
 * (device pointers; nx, ny multiples of factor).  Synchronous on `stream`
 * (cudaStream_t or NULL). */
int fv_coarsen(const float* fine, int planes, int ny, int nx, int factor, float* coarse, void* stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of solve requests
 *
 * The request/response pair of the serving loop is named fv_submit /
 * fv_poll (not submit / poll: a C symbol `poll` exported by a shared library
 * would interpose the C library's poll(2) for the whole process).
 * ------------------------------------------------------------------------- */

/* One solve request: a single member on an nx x ny periodic unit square,
 * advanced nsteps SSP-RK2 steps with the adaptive CFL time step at Courant
 * number cfl.  eq: FV_EQ_SWE or FV_EQ_EULER; learned != 0 uses the server's
 * network (shallow water only; nx must be 8, 16, 32, 64 or a multiple of
 * 128).  q0: host [C][ny][nx], copied at submission. */
typedef struct {
  int eq;
  int learned;
  int nx, ny;
  long nsteps;
  double cfl;
  const float* q0;
} fv_request;

/* A server with a device-memory budget for resident request states and at
 * most max_slots requests on the device at once; net (may be NULL, borrowed)
 * serves learned requests.  A worker thread admits requests in arrival order
 * as slots and memory free up, keeps admitted states resident, and advances
 * every admitted request by graph-replayed chunks on its own stream, so
 * requests that arrive while others run overlap on the GPU. */
int fv_server_create(size_t hbm_budget_bytes, int max_slots, const fv_net* net, fv_server** out);

/* Stop the worker (requests still running end with FV_ETIMEOUT) and free
 * everything, including results not yet polled. */
int fv_server_destroy(fv_server* s);

/* Queue a request; *ticket identifies it.  FV_EBUSY if its device-memory
 * footprint exceeds the whole budget (it could never be admitted),
 * FV_EINVAL for a malformed request. */
int fv_submit(fv_server* s, const fv_request* r, unsigned long long* ticket);

/* A learned request whose state becomes non-physical is rerun from its
 * initial state with the plain MUSCL-minmod step (the learned step's
 * fallback); fv_server_stats counts these. */

/* FV_PENDING while the request waits or runs.  Once done: copies the final
 * state to q_out (host [C][ny][nx], may be NULL), the submission-to-
 * completion latency to *latency_s, forgets the ticket and returns FV_OK or
 * the request's error (FV_EUNSTABLE, FV_ECUDA, ...).  FV_ENOTFOUND for an
 * unknown or already collected ticket. */
int fv_poll(fv_server* s, unsigned long long ticket, float* q_out, double* latency_s);

/* Requests on the device, requests waiting, device bytes reserved, learned
 * requests that fell back to the plain step so far (any pointer may be NULL). */
int fv_server_stats(fv_server* s, int* active, int* pending, size_t* used_bytes,
                    long long* fallbacks);

/* ---------------------------------------------------------------------------
 * Training: taped learned rollout, rollout loss (Eq. 2.28), backward, Adam
 * ------------------------------------------------------------------------- */
typedef struct fv_tape fv_tape;

/* A tape for T learned SSP-RK2 steps of B shallow-water members on an
 * nx x ny periodic unit square with a fixed dt, gravity g and positivity
 * threshold h_min = hmin_frac * (mean depth of each member's q0; unused by
 * a face-state network).  The tape owns device buffers for every stage
 * input, the CNN activations and the coefficients (or side states).  net is
 * borrowed and must outlive the tape. */
int fv_tape_create(fv_net* net, int B, int ny, int nx, int T, double dt, double g, double hmin_frac,
                   fv_tape** out);
int fv_tape_destroy(fv_tape* t);

/* Run the T steps from q0 (device [B][3][ny][nx]) with the network's current
 * parameters, recording the tape; snaps (device [T][B][3][ny][nx], may be
 * NULL) receives q_1 .. q_T.  Synchronous; FV_EUNSTABLE if a state went
 * non-physical. */
int fv_tape_forward(fv_tape* t, const float* q0, float* snaps);

/* Eq. 2.28 over the recorded rollout: loss = sum_{t=1..T} sum_c
 * mean_{members, cells} ((q_t - target_t) / scale_c)^2 with targets (device
 * [T][B][3][ny][nx]) and scale3 (host [3]).  Keeps d loss / d q_t on the
 * tape for fv_tape_backward. */
int fv_tape_loss(fv_tape* t, const float* targets, const float* scale3, double* loss);

/* Reverse pass through the recorded rollout.  dsnaps: device [T][B][3][ny][nx]
 * cotangents of q_1 .. q_T, or NULL for the gradient of the last
 * fv_tape_loss.  Adds the parameter gradient to dparams (device
 * [fv_net_num_params(net)]); dq0 (device [B][3][ny][nx], may be NULL) receives the
 * cotangent of q0.  Cotangents between CNN layers are BF16 (tensor-core
 * operands); everything else is FP32. */
int fv_tape_backward(fv_tape* t, const float* dsnaps, float* dparams, float* dq0);

/* One Adam step (bias-corrected; moments kept in the network) with the
 * gradient grad (device [fv_net_num_params(n)]); step counts from 1.  Repacks
 * the tensor-core weights. */
int stencil_net_adam_step(fv_net* n, const float* grad, int step, double lr, double b1, double b2,
                          double eps);

#ifdef __cplusplus
}
#endif
#endif /* FV_H_ */
