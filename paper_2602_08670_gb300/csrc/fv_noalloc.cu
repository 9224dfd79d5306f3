// fv_noalloc.cu — FP64 diagnostics without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a host
// loop that received its whole device-memory budget up front, code in an
// allocation-free region (a real-time loop, a host callback) where the
// implicit synchronisation and possible failure of cudaMalloc are not
// acceptable, or a framework that hands out all device memory through its own
// pool.  For them fv_diagnostics_noalloc() computes the same sums as
// fv_diagnostics() on a state the caller already holds, with the reduction
// scratch in a fixed-size array of this file that every GPU loading the
// library keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "fv_common.cuh"
#include "fv_kernels.h"

namespace {

// Largest batch * (C + 1) the scratch holds: 64 Euler members (C + 1 = 5) or
// 80 shallow-water members (C + 1 = 4).
constexpr int kMaxSlots = 320;
constexpr int kPartialsPerSlot = 256;   // blocks of the partial-sum kernel

static __device__ __align__(256) double g_diag_partials[kMaxSlots * kPartialsPerSlot];
static __device__ __align__(256) double g_diag_result[kMaxSlots];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_partials_ptr[kMaxDevices] = {};
double* g_result_ptr[kMaxDevices] = {};

// Device addresses of the two arrays on the current device, looked up once
// per device with that device current.
int scratch_for_current_device(double** partials, double** result) {
  int dev = 0;
  FV_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fvh::fail(FV_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    void* r = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_diag_partials);
    if (e != cudaSuccess) return fvh::cuda_fail(e, "cudaGetSymbolAddress(diagnostics scratch)");
    e = cudaGetSymbolAddress(&r, g_diag_result);
    if (e != cudaSuccess) return fvh::cuda_fail(e, "cudaGetSymbolAddress(diagnostics result)");
    g_partials_ptr[dev] = static_cast<double*>(p);
    g_result_ptr[dev] = static_cast<double*>(r);
  }
  *partials = g_partials_ptr[dev];
  *result = g_result_ptr[dev];
  return FV_OK;
}

}  // namespace

extern "C" int fv_diagnostics_noalloc(const float* q, int eq, int batch, int ny, int nx, double lx,
                                      double ly, double phys, double* sums, int sums_loc,
                                      void* stream) {
  if (!q || !sums) return fvh::fail(FV_EINVAL, "null argument");
  if (eq != FV_EQ_SWE && eq != FV_EQ_EULER) return fvh::fail(FV_EINVAL, "unknown equation set");
  if (batch < 1 || ny < 1 || nx < 1 || !(lx > 0) || !(ly > 0))
    return fvh::fail(FV_EINVAL, "bad sizes");
  if (sums_loc != FV_HOST && sums_loc != FV_DEVICE) return fvh::fail(FV_EINVAL, "bad sums location");
  const int C = eq == FV_EQ_SWE ? 3 : 4;
  if ((long long)batch * (C + 1) > kMaxSlots)
    return fvh::fail(FV_EINVAL, "fv_diagnostics_noalloc: batch * (variables + 1) exceeds the fixed "
                                "scratch of 320 slots (at most 80 shallow-water or 64 Euler members)");
  double *partials = nullptr, *result = nullptr;
  int rc = scratch_for_current_device(&partials, &result);
  if (rc != FV_OK) return rc;
  fvk::Geom g{};
  g.nx = nx;
  g.ny = ny;
  g.B = batch;
  g.C = C;
  g.eq = eq == FV_EQ_SWE ? fvk::SWE : fvk::EULER;
  g.dx = lx / nx;
  g.dy = ly / ny;
  g.phys = (float)phys;
  g.phys_d = phys;
  if (fvk::diag_partials_size(g) > (long long)kMaxSlots * kPartialsPerSlot)
    return fvh::fail(FV_EINVAL, "fv_diagnostics_noalloc: reduction does not fit the fixed scratch");
  // every partial slot the final reduction reads is written by this call's
  // partial kernel first, so nothing needs clearing between calls
  cudaStream_t s = (cudaStream_t)stream;
  double* out = sums_loc == FV_DEVICE ? sums : result;
  FV_CUDA_TRY(fvk::launch_diagnostics(g, q, partials, out, s));
  if (sums_loc == FV_HOST) {
    FV_CUDA_TRY(cudaMemcpyAsync(sums, result, sizeof(double) * batch * (C + 1), cudaMemcpyDeviceToHost, s));
    FV_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return FV_OK;
}
