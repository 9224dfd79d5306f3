// fv_util.cu — coarse graining of cell averages.
//
// The coarse cell average of a factor x factor block of fine cell averages is
// their mean (Section 2.5.1: training targets are high-resolution runs
// coarsened to the low resolution).  HBM-bound: each fine value is read once,
// each coarse value written once.
#include <cuda_runtime.h>

#include "fv_common.cuh"

namespace {

// One thread per coarse cell; a warp covers consecutive coarse x, so each
// fine row segment it reads is contiguous.
__global__ void coarsen_kernel(const float* fine, float* coarse, int nxc, int nyc, int factor,
                               long long planes) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long per_plane = (long long)nxc * nyc;
  if (t >= planes * per_plane) return;
  const long long p = t / per_plane;
  const int c = (int)(t - p * per_plane);
  const int yc = c / nxc, xc = c - yc * nxc;
  const int nxf = nxc * factor;
  const float* src = fine + p * per_plane * factor * factor + (long long)yc * factor * nxf + xc * factor;
  double s = 0.0;
  for (int j = 0; j < factor; ++j)
    for (int i = 0; i < factor; ++i) s += src[(long long)j * nxf + i];
  coarse[t] = (float)(s / (double)(factor * factor));
}

}  // namespace

extern "C" int fv_coarsen(const float* fine, int planes, int ny, int nx, int factor, float* coarse,
                          void* stream) {
  if (!fine || !coarse || planes < 1 || factor < 1 || nx % factor || ny % factor)
    return fvh::fail(FV_EINVAL, "fv_coarsen: bad arguments (nx, ny must be multiples of factor)");
  const int nxc = nx / factor, nyc = ny / factor;
  const long long n = (long long)planes * nxc * nyc;
  coarsen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(fine, coarse, nxc, nyc,
                                                                                 factor, planes);
  FV_CUDA_TRY(cudaGetLastError());
  FV_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  return FV_OK;
}
