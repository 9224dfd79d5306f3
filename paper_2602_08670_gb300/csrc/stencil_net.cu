// stencil_net.cu — the learned-stencil CNN on tcgen05 tensor cores.
//
// Each 3x3 periodic convolution is an implicit GEMM: M = 128 consecutive
// cells of one member, N = output channels, K = 9 taps x input channels.  A
// CTA stages the input cells its tile needs (with periodic wrap) in shared
// memory in the K-major canonical layout [channel group][position][8 BF16],
// arranged so that for every tap the 128 shifted input rows are contiguous
// positions: one shared-memory descriptor per (tap, 16-channel step) then
// addresses them directly, and 9 x (C_in / 16) tcgen05.mma instructions
// accumulate the tile in TMEM (FP32).  The epilogue reads TMEM, adds the
// bias and either applies ReLU and stores BF16 activations, or normalises
// each 3-tap stencil (w = e_centre + r - mean(r)) and stores the FP32
// coefficients.  The first layer reads the FP32 state and normalises it
// (x = (q - mean) / std) while staging.  The face-state network (third
// approach) uses the same kernel with a GeLU epilogue on the hidden layers
// and a side-state epilogue (Softplus depths, de-normalised momenta) on the
// last one.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fv_common.cuh"
#include "stencil_net.cuh"
#include "tc_common.cuh"

namespace snk {

ParamLayout param_layout(int kind) {
  ParamLayout L{};
  const int cout[4] = {HID, HID, HID, kind == NET_FACE ? N_OUT_FACE : N_OUT};
  const int cin[4] = {C_IN, HID, HID, HID};
  int off = 0;
  for (int l = 0; l < 4; ++l) {
    L.cout[l] = cout[l];
    L.cin[l] = cin[l];
    L.w[l] = off;
    off += cout[l] * cin[l] * 9;
    L.b[l] = off;
    off += cout[l];
  }
  return L;
}

int n_params(int kind) { return kind == NET_FACE ? N_PARAMS_FACE : N_PARAMS; }

bool grid_supported(int nx) { return nx % TILE == 0 || nx == 8 || nx == 16 || nx == 32 || nx == 64; }

namespace {

constexpr int NT = 128;                 // threads per CTA (4 warps = 128 TMEM lanes)
constexpr int RW = TILE + 2;            // row mode: staged row width (1-cell halo each side)
constexpr int NPOS_ROW = 3 * RW;        // row mode: 3 rows
constexpr int NPOS_MAX = 3 * (TILE + 2 * 64);   // strip mode with nx <= 64 (CUDA-core dW)
constexpr int GSLOT = 10;               // grouped mode: 8 cells + the x-neighbour on each side
constexpr uint32_t WAIT_ITERS = 1u << 22;

enum { IN_STATE = 0, IN_ACT = 1 };
enum { OUT_RELU = 0, OUT_W = 1, OUT_RAW = 2, OUT_MASK = 3, OUT_GELU = 4, OUT_SIDES = 5, OUT_SIDES_RAW = 6,
       OUT_GELU_GRAD = 7, OUT_DQ = 8 };

struct ConvArgs {
  const float* q;          // IN_STATE: [B][3][plane]
  const uint16_t* x;       // IN_ACT: [B][4][plane][8]
  const uint16_t* wpk;     // [9][CG][N][8]
  const float* bias;
  uint16_t* y;             // OUT_RELU: [B][4][plane][8]
  float* w;                // OUT_W / OUT_RAW: [B][36][plane]; OUT_SIDES(_RAW): [B][12][plane];
                           // OUT_DQ: dq [B][3][plane], added to
  const uint16_t* mask;    // OUT_MASK: activation [B][4][plane][8]; output kept where it is > 0
  uint16_t* z;             // OUT_GELU: pre-activations out (if non-null); OUT_GELU_GRAD: in
  float mean0, mean1, mean2, rstd0, rstd1, rstd2;
  float std1, std2;        // OUT_SIDES: momentum de-normalisation
  int nx, ny;
  long long plane;
  unsigned* err;
};

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// i in [-n, 2n): the periodic index in [0, n).
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ int floordiv(int a, int b) {
  const int q = a / b;
  return (a % b != 0 && (a < 0) != (b < 0)) ? q - 1 : q;
}

// Staged input positions of the CUDA-core weight gradient: row mode (nx a
// multiple of the tile) 3 rows of TILE + 2 cells, strip mode (nx <= 64) 3
// x-shifted strips of TILE + 2 nx.
template <bool ROW>
constexpr int npos_of() { return ROW ? NPOS_ROW : NPOS_MAX; }

// Staged input positions of the convolution: row mode as above; grouped mode
// (nx <= 64 dividing the tile, which then covers TILE / nx whole rows) keeps
// every run of 8 cells of the rows y0 - 1 .. y0 + TILE / nx with its two
// periodic x-neighbours, 10 positions per run.  The MMA rows of a tap (dy,
// dx) are then 8-row groups 10 positions apart: one descriptor with a
// 160-byte group stride covers the tile for every tap, with a third of the
// staging of three x-shifted strips.
//
// A CTA convolves TPC = 1 or 2 tiles: in row mode the tiles at the same
// columns of rows y0 and y0 + 1 (4 staged rows for both), in grouped mode
// two consecutive tiles (their rows and the two rows around them).  The
// pair shares the staged rows between them and one load of the weights.
template <bool ROW, int TPC = 1>
constexpr int conv_np() { return ROW ? (TPC + 2) * RW : (TPC * TILE / 8 + 2 * 64 / 8) * GSLOT; }

template <int CG, int N, bool ROW, int TPC = 1>
constexpr int conv_smem_bytes() {
  return CG * conv_np<ROW, TPC>() * 16 + 9 * CG * N * 16 + 64;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// GeLU, x Phi(x) with Phi(x) = (1 + erf(x / sqrt 2)) / 2, for two values at
// once.  erf is Hastings' approximation (Abramowitz & Stegun 7.1.28): for
// t >= 0, erf(t) = 1 - r with r = (1 + a1 t + ... + a6 t^6)^-16 and
// |error| <= 3e-7 (1.7e-6 when evaluated in FP32, the 16th power amplifying
// the rounding of the polynomial).  For x < 0, Phi = r / 2 directly, without
// the cancellation of 1 - erf.  Packed FP32x2 arithmetic and one reciprocal
// per value: a third of the instructions of the library erf, which bounded
// the GeLU layers.  Its absolute error is far below the BF16 rounding of
// the activations.
__device__ __forceinline__ float2 gelu2(float2 x) {
  const float2 t = make_float2(fabsf(x.x) * 0.70710678118654752f, fabsf(x.y) * 0.70710678118654752f);
  float2 p = fvk::vfma(t, fvk::vsplat<float2>(0.0000430638f), fvk::vsplat<float2>(0.0002765672f));
  p = fvk::vfma(p, t, fvk::vsplat<float2>(0.0001520143f));
  p = fvk::vfma(p, t, fvk::vsplat<float2>(0.0092705272f));
  p = fvk::vfma(p, t, fvk::vsplat<float2>(0.0422820123f));
  p = fvk::vfma(p, t, fvk::vsplat<float2>(0.0705230784f));
  p = fvk::vfma(p, t, fvk::vsplat<float2>(1.f));
  p = fvk::vmul(p, p);
  p = fvk::vmul(p, p);
  p = fvk::vmul(p, p);
  p = fvk::vmul(p, p);                                        // p^16
  const float2 r = make_float2(fvk::vrcp(p.x), fvk::vrcp(p.y));   // 1 - erf(t)
  const float phi0 = x.x >= 0.f ? fmaf(-0.5f, r.x, 1.f) : 0.5f * r.x;
  const float phi1 = x.y >= 0.f ? fmaf(-0.5f, r.y, 1.f) : 0.5f * r.y;
  return fvk::vmul(x, make_float2(phi0, phi1));
}

// Softplus, log(1 + e^x) = max(x, 0) + log(1 + e^-|x|).
__device__ __forceinline__ float softplus(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }

// d GeLU / dx = Phi(x) + x phi(x), phi the standard normal density.
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::smem_u32(smem)), "l"(gmem)
               : "memory");
}

// Stage the input positions of the 128-cell tile at p0 of member b into sA
// ([CG][NP][16 B], row or grouped mode, see conv_np).  Activations arrive by
// cp.async (the caller commits and waits); the state is normalised and
// stored directly.  Every offset lies within one period of the grid, so one
// compare-and-select wraps it; a power-of-two width divides by a shift.
template <int CG, int IN, bool ROW, int TPC = 1>
__device__ __forceinline__ void conv_stage(const ConvArgs& a, uint8_t* sA, int b, int p0, int tid) {
  constexpr int NP = conv_np<ROW, TPC>();
  const int nx = a.nx, ny = a.ny;
  const int lg = (nx & (nx - 1)) == 0 ? __ffs(nx) - 1 : -1;
  const int y0 = lg >= 0 ? p0 >> lg : p0 / nx, x0 = p0 - y0 * nx;
  const int gpr = nx >> 3;                             // grouped mode: runs of 8 per row
  const int npos = ROW ? (TPC + 2) * RW : (TPC * TILE / 8 + 2 * gpr) * GSLOT;
  if constexpr (IN == IN_STATE) {
    // the state: every load of this thread issued before the first use
    constexpr int IT = (NP + NT - 1) / NT;
    const float* qb = a.q + (long long)b * 3 * a.plane;
    float h[IT][3];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int n = tid + it * NT;
      if (n < npos) {
        int yy, xx;
        if (ROW) {
          const int dyi = n / RW, xi = n - dyi * RW;
          yy = wrap1(y0 - 1 + dyi, ny);
          xx = wrap1(x0 - 1 + xi, nx);
        } else {
          const int run = n / GSLOT, sl = n - run * GSLOT;
          const int ry = run / gpr, gi = run - ry * gpr;
          yy = wrap1(y0 - 1 + ry, ny);
          xx = wrap1(8 * gi - 1 + sl, nx);
        }
        const long long cell = (long long)yy * nx + xx;
        h[it][0] = __ldg(qb + cell);
        h[it][1] = __ldg(qb + a.plane + cell);
        h[it][2] = __ldg(qb + 2 * a.plane + cell);
      }
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int n = tid + it * NT;
      if (n < npos) {
        const float h0 = (h[it][0] - a.mean0) * a.rstd0;
        const float h1 = (h[it][1] - a.mean1) * a.rstd1;
        const float h2 = (h[it][2] - a.mean2) * a.rstd2;
        *reinterpret_cast<uint4*>(sA + n * 16) = make_uint4(pack_bf16x2(h0, h1), pack_bf16x2(h2, 0.f), 0u, 0u);
#pragma unroll
        for (int g = 1; g < CG; ++g) *reinterpret_cast<uint4*>(sA + (g * NP + n) * 16) = make_uint4(0, 0, 0, 0);
      }
    }
  } else {
    // activations: 16-byte records by cp.async
    for (int n = tid; n < npos; n += NT) {
      int yy, xx;
      if (ROW) {
        const int dyi = n / RW, xi = n - dyi * RW;
        yy = wrap1(y0 - 1 + dyi, ny);
        xx = wrap1(x0 - 1 + xi, nx);
      } else {
        const int run = n / GSLOT, sl = n - run * GSLOT;
        const int ry = run / gpr, gi = run - ry * gpr;  // x0 = 0: the tile starts a row
        yy = wrap1(y0 - 1 + ry, ny);
        xx = wrap1(8 * gi - 1 + sl, nx);
      }
      const long long cell = (long long)yy * nx + xx;
#pragma unroll
      for (int g = 0; g < CG; ++g)
        cp_async16(sA + (g * NP + n) * 16, a.x + (((long long)b * CG + g) * a.plane + cell) * 8);
    }
  }
}

// Epilogue of one tile: thread m (TMEM lane m) finishes cell `cell` of
// member b from the accumulator at lane_addr.
template <int N, int OUT>
__device__ __forceinline__ void conv_epilogue(const ConvArgs& a, int b, long long cell, uint32_t lane_addr) {
  if constexpr (OUT == OUT_MASK) {
    // backward through ReLU: cotangent of the layer input, zero where the
    // stored activation is zero (BF16 out, 32 channels)
    float v[32];
    tc::tmem_ld32(lane_addr, v);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const uint4 mk = *reinterpret_cast<const uint4*>(a.mask + (((long long)b * 4 + g) * a.plane + cell) * 8);
      const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
      uint32_t pk[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c0 = 8 * g + 2 * j;
        const bool p0 = (mw[j] & 0x7FFFu) != 0 && !(mw[j] & 0x8000u);
        const bool p1 = ((mw[j] >> 16) & 0x7FFFu) != 0 && !((mw[j] >> 16) & 0x8000u);
        pk[j] = pack_bf16x2(p0 ? v[c0] : 0.f, p1 ? v[c0 + 1] : 0.f);
      }
      *reinterpret_cast<uint4*>(a.y + (((long long)b * 4 + g) * a.plane + cell) * 8) =
          make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  } else if constexpr (OUT == OUT_GELU_GRAD) {
    // backward through GeLU: cotangent of the layer input times GeLU' of
    // the stored pre-activation (BF16 out, 32 channels)
    float v[32];
    tc::tmem_ld32(lane_addr, v);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const uint4 zk = *reinterpret_cast<const uint4*>(a.z + (((long long)b * 4 + g) * a.plane + cell) * 8);
      const uint32_t zw[4] = {zk.x, zk.y, zk.z, zk.w};
      uint32_t pk[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c0 = 8 * g + 2 * j;
        const float z0 = __uint_as_float(zw[j] << 16), z1 = __uint_as_float(zw[j] & 0xFFFF0000u);
        pk[j] = pack_bf16x2(v[c0] * gelu_grad(z0), v[c0 + 1] * gelu_grad(z1));
      }
      *reinterpret_cast<uint4*>(a.y + (((long long)b * 4 + g) * a.plane + cell) * 8) =
          make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  } else if constexpr (OUT == OUT_RELU || OUT == OUT_GELU) {
    float v[32];
    tc::tmem_ld32(lane_addr, v);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      uint32_t pk[4], pz[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c0 = 8 * g + 2 * j;
        const float z0 = v[c0] + a.bias[c0], z1 = v[c0 + 1] + a.bias[c0 + 1];
        if constexpr (OUT == OUT_RELU) {
          pk[j] = pack_bf16x2(fmaxf(z0, 0.f), fmaxf(z1, 0.f));
        } else {
          const float2 gz = gelu2(make_float2(z0, z1));
          pk[j] = pack_bf16x2(gz.x, gz.y);
          pz[j] = pack_bf16x2(z0, z1);
        }
      }
      *reinterpret_cast<uint4*>(a.y + (((long long)b * 4 + g) * a.plane + cell) * 8) =
          make_uint4(pk[0], pk[1], pk[2], pk[3]);
      if constexpr (OUT == OUT_GELU) {
        if (a.z)
          *reinterpret_cast<uint4*>(a.z + (((long long)b * 4 + g) * a.plane + cell) * 8) =
              make_uint4(pz[0], pz[1], pz[2], pz[3]);
      }
    }
  } else if constexpr (OUT == OUT_DQ) {
    // first layer's dX (3 channels of the normalised state): dq += dx / std
    float v[16];
    tc::tmem_ld16(lane_addr, v);
    float* d = a.w + (long long)b * 3 * a.plane + cell;
    d[0] += v[0] * a.rstd0;
    d[a.plane] += v[1] * a.rstd1;
    d[2 * a.plane] += v[2] * a.rstd2;
  } else if constexpr (OUT == OUT_SIDES || OUT == OUT_SIDES_RAW) {
    // side states of the face-state network: channel 3 side + var
    float v[16];
    tc::tmem_ld16(lane_addr, v);
    float* sb = a.w + (long long)b * N_OUT_FACE * a.plane + cell;
#pragma unroll
    for (int k = 0; k < N_OUT_FACE; ++k) {
      const float r = v[k] + a.bias[k];
      float o = r;
      if constexpr (OUT == OUT_SIDES) {
        const int var = k % 3;
        o = var == 0 ? softplus(r) : (var == 1 ? fmaf(a.std1, r, a.mean1) : fmaf(a.std2, r, a.mean2));
      }
      sb[k * a.plane] = o;
    }
  } else {
    float v[32], v2[16];
    tc::tmem_ld32(lane_addr, v);
    tc::tmem_ld16(lane_addr + 32, v2);
    float r[N_OUT];
#pragma unroll
    for (int k = 0; k < 32; ++k) r[k] = v[k] + a.bias[k];
#pragma unroll
    for (int k = 32; k < N_OUT; ++k) r[k] = v2[k - 32] + a.bias[k];
    float* wb = a.w + (long long)b * N_OUT * a.plane + cell;
    if constexpr (OUT == OUT_RAW) {
#pragma unroll
      for (int k = 0; k < N_OUT; ++k) wb[k * a.plane] = r[k];
    } else {
#pragma unroll
      for (int s = 0; s < N_OUT / 3; ++s) {
        const float mean = (r[3 * s] + r[3 * s + 1] + r[3 * s + 2]) * (1.f / 3.f);
        wb[(3 * s) * a.plane] = r[3 * s] - mean;
        wb[(3 * s + 1) * a.plane] = 1.f + (r[3 * s + 1] - mean);
        wb[(3 * s + 2) * a.plane] = r[3 * s + 2] - mean;
      }
    }
  }
}

template <int CG, int N, int IN, int OUT, bool ROW, int TPC>
__global__ void __launch_bounds__(NT) conv_kernel(ConvArgs a) {
  constexpr int NP = conv_np<ROW, TPC>();
  constexpr uint32_t NCOLS = TPC * N <= 32 ? 32u : (TPC * N <= 64 ? 64u : 128u);
  static_assert(TPC * N <= 128, "accumulator columns");
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;                                   // [CG][NP][16 B]
  uint8_t* sB = smem + CG * NP * 16;                    // [9][CG][N][16 B]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + 9 * CG * N * 16);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x;
  constexpr bool rowmode = ROW;
  const int gpr = a.nx >> 3;
  // the CTA's tiles: p0 of tile u is p0 + u * tile_step
  const long long units_per_member = a.plane / (TILE * TPC);
  const int b = (int)(blockIdx.x / units_per_member);
  const int unit = (int)(blockIdx.x - (long long)b * units_per_member);
  int p0, tile_step;
  if (ROW && TPC == 2) {
    const int tpr = a.nx / TILE;                        // tiles per row
    const int y2 = unit / tpr, xt = unit - y2 * tpr;
    p0 = 2 * y2 * a.nx + xt * TILE;
    tile_step = a.nx;                                   // the next row
  } else {
    p0 = unit * TILE * TPC;
    tile_step = TILE;
  }

  if (tid < 32) tc::tmem_alloc(tslot, NCOLS);
  if (tid == 0) tc::mbar_init(mbar, 1);

  // weights: 9 * CG * N chunks of 16 bytes
  for (int i = tid; i < 9 * CG * N; i += NT) cp_async16(sB + i * 16, a.wpk + i * 8);

  conv_stage<CG, IN, ROW, TPC>(a, sA, b, p0, tid);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(TILE, N);
    const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
    for (int u = 0; u < TPC; ++u) {
      bool acc = false;
#pragma unroll 1
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        // row mode: 8-row groups 128 B apart, tile u one staged row down;
        // grouped mode: 160 B apart, tile u 16 runs on
        const int start = rowmode ? (u + 1 + dy) * RW + (1 + dx) : (u * (TILE / 8) + (1 + dy) * gpr) * GSLOT + (1 + dx);
        constexpr uint32_t sbo = rowmode ? 128u : 16u * GSLOT;
#pragma unroll
        for (int ks = 0; ks < CG / 2; ++ks) {
          const uint64_t ad = tc::sdesc(a0 + (uint32_t)((2 * ks * NP + start) * 16), NP * 16, sbo);
          const uint64_t bd = tc::sdesc(b0 + (uint32_t)(((tap * CG + 2 * ks) * N) * 16), N * 16, 128);
          tc::mma_bf16(tmem + (uint32_t)(u * N), ad, bd, idesc, acc);
          acc = true;
        }
      }
    }
    tc::mma_commit(mbar);
  }
  const bool ok = tc::mbar_wait_bounded(mbar, 0, WAIT_ITERS);
  if (!ok && tid == 0) atomicOr(a.err, 1u);
  tc::fence_after_sync();

  if (ok) {
    const int w = tid >> 5;
    const int m = tid;                                   // TMEM lane = tile row
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * w) << 16);
#pragma unroll
    for (int u = 0; u < TPC; ++u)
      conv_epilogue<N, OUT>(a, b, (long long)p0 + u * tile_step + m, lane_addr + (uint32_t)(u * N));
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid < 32) tc::tmem_dealloc(tmem, NCOLS);
}

// FP32 master parameters -> BF16 operand layouts.
//   forward  wf[l][tap][g][n][k8] = W_l[n][8g + k8][ky][kx]
//   backward wb[l][tap][g][n][k8] = W_l[8g + k8][n][2 - ky][2 - kx]   (l >= 1; l = 0 with
//            N = 16, n < 3 the state's channels, the rest zero)
// The row-pipelined operands (w1g, wpair, w4ring) exist for the stencil
// network only; they are skipped when null.  n_last: N of the last layer.
__global__ void repack_kernel(const float* params, ParamLayout L, uint16_t* wf0, uint16_t* wf1,
                              uint16_t* wf2, uint16_t* wf3, uint16_t* wb0, uint16_t* wb1, uint16_t* wb2,
                              uint16_t* wb3, uint16_t* w1g, uint16_t* wp1, uint16_t* wp2,
                              uint16_t* w4r, int n_last) {
  uint16_t* wf[4] = {wf0, wf1, wf2, wf3};
  uint16_t* wb[4] = {wb0, wb1, wb2, wb3};
  const int cgs[4] = {CG_IN0, CG_HID, CG_HID, CG_HID};
  const int ns[4] = {HID, HID, HID, n_last};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (w1g && i < W1G_ELEMS) {
    // w1g[ky][g][n][k8] = W_1[n][var][ky][kx] with 8 g + k8 = 3 kx + var
    const int k8 = i % 8, n = (i / 8) % HID, g = (i / (8 * HID)) % 2, ky = i / (16 * HID);
    const int c = 8 * g + k8;
    float v = 0.f;
    if (c < 3 * C_IN) v = params[L.w[0] + ((n * C_IN + c % 3) * 3 + ky) * 3 + c / 3];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    w1g[i] = *reinterpret_cast<const uint16_t*>(&h);
  }
  if (w4r && i < W4R_ELEMS) {
    // w4ring[kx][g][n][k8]: block n / 24 holds the tap ky = 2, 1, 0, 2, 1; row
    // r = n % 24 = 2 s + j the difference W_4[3 s + j] - W_4[3 s + 2]
    const int k8 = i % 8, n = (i / 8) % W4R_ROWS, g = (i / (8 * W4R_ROWS)) % CG_HID,
              kx = i / (8 * W4R_ROWS * CG_HID);
    const int ci = 8 * g + k8;
    float v = 0.f;
    if (n < 5 * W4R_BLOCK && ci < L.cin[3]) {
      const int blk = n / W4R_BLOCK, r = n % W4R_BLOCK;
      const int ky = blk == 2 ? 0 : (blk == 1 || blk == 4 ? 1 : 2);
      const int s = r / 2, j = r % 2;
      const int ca = 3 * s + j, cc = 3 * s + 2;
      v = params[L.w[3] + ((ca * L.cin[3] + ci) * 3 + ky) * 3 + kx] -
          params[L.w[3] + ((cc * L.cin[3] + ci) * 3 + ky) * 3 + kx];
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    w4r[i] = *reinterpret_cast<const uint16_t*>(&h);
  }
  uint16_t* wp[3] = {nullptr, wp1, wp2};
  for (int l = 1; l < 3; ++l) {
    // [ky = 0: kx][g][n][k8], then [kx][g][ky = 2 | ky = 1][k8]
    const int N = HID;
    const int part0 = 3 * CG_HID * N * 8;
    if (wp[l] && i < 9 * CG_HID * N * 8) {
      int kx, g, n, k8, ky;
      if (i < part0) {
        k8 = i % 8;
        n = (i / 8) % N;
        g = (i / (8 * N)) % CG_HID;
        kx = i / (8 * N * CG_HID);
        ky = 0;
      } else {
        const int j = i - part0;
        k8 = j % 8;
        const int n2 = (j / 8) % (2 * N);
        g = (j / (16 * N)) % CG_HID;
        kx = j / (16 * N * CG_HID);
        ky = n2 < N ? 2 : 1;
        n = n2 % N;
      }
      const int ci = 8 * g + k8, co = n;
      float v = 0.f;
      if (ci < L.cin[l] && co < L.cout[l]) v = params[L.w[l] + ((co * L.cin[l] + ci) * 3 + ky) * 3 + kx];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      wp[l][i] = *reinterpret_cast<const uint16_t*>(&h);
    }
  }
  for (int l = 0; l < 4; ++l) {
    const int CG = cgs[l], N = ns[l];
    const int total = 9 * CG * N * 8;
    if (i < total) {
      const int k8 = i % 8, n = (i / 8) % N, g = (i / (8 * N)) % CG, tap = i / (8 * N * CG);
      const int ci = 8 * g + k8, co = n;
      float v = 0.f;
      if (ci < L.cin[l] && co < L.cout[l]) v = params[L.w[l] + ((co * L.cin[l] + ci) * 3 + tap / 3) * 3 + tap % 3];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      wf[l][i] = *reinterpret_cast<const uint16_t*>(&h);
    }
    if (wb[l]) {
      // dX of layer l: K = its output channels (groups of 8), N = its inputs
      // (32; 16 for the 3 state channels of layer 1)
      const int CGo = (L.cout[l] + 7) / 8 + ((L.cout[l] + 7) / 8) % 2;   // even number of groups
      const int Nb = l == 0 ? DQ_N : HID;
      const int totb = 9 * CGo * Nb * 8;
      if (i < totb) {
        const int k8 = i % 8, n = (i / 8) % Nb, g = (i / (8 * Nb)) % CGo, tap = i / (8 * Nb * CGo);
        const int co = 8 * g + k8, ci = n;
        const int fy = 2 - tap / 3, fx = 2 - tap % 3;
        float v = 0.f;
        if (co < L.cout[l] && ci < L.cin[l]) v = params[L.w[l] + ((co * L.cin[l] + ci) * 3 + fy) * 3 + fx];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        wb[l][i] = *reinterpret_cast<const uint16_t*>(&h);
      }
    }
  }
}

template <int CG, int N, int IN, int OUT, bool ROW, int TPC>
cudaError_t launch_conv_t(const ConvArgs& a, int B, cudaStream_t s) {
  constexpr int smem = conv_smem_bytes<CG, N, ROW, TPC>();
  auto kern = conv_kernel<CG, N, IN, OUT, ROW, TPC>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long ctas = (long long)B * (a.plane / (TILE * TPC));
  kern<<<(unsigned)ctas, NT, smem, s>>>(a);
  return cudaGetLastError();
}

// Row mode (nx a multiple of the tile) stages rows; grouped mode serves the
// narrow grids.  Two tiles per CTA where the grid pairs them (an even number
// of rows in row mode, whole 256-cell pairs in grouped mode).
template <int CG, int N, int IN, int OUT>
cudaError_t launch_conv(const ConvArgs& a, int B, cudaStream_t s) {
  if (a.nx % TILE == 0) {
    if (a.ny % 2 == 0) return launch_conv_t<CG, N, IN, OUT, true, 2>(a, B, s);
    return launch_conv_t<CG, N, IN, OUT, true, 1>(a, B, s);
  }
  if (a.plane % (2 * TILE) == 0) return launch_conv_t<CG, N, IN, OUT, false, 2>(a, B, s);
  return launch_conv_t<CG, N, IN, OUT, false, 1>(a, B, s);
}

}  // namespace

int backward_groups(int cout) {
  const int g = (cout + 7) / 8;
  return g + (g % 2);
}

cudaError_t repack(Net& net, cudaStream_t s) {
  const int maxn = 9 * CG_HID * N_OUT_PAD * 8 > 9 * 6 * HID * 8 ? 9 * CG_HID * N_OUT_PAD * 8 : 9 * 6 * HID * 8;
  static_assert(W4R_ELEMS <= 9 * CG_HID * N_OUT_PAD * 8, "repack grid covers the layer-4 ring weights");
  const ParamLayout Lk = param_layout(net.kind);
  repack_kernel<<<(maxn + 255) / 256, 256, 0, s>>>(net.params, Lk, net.wf[0], net.wf[1], net.wf[2],
                                                   net.wf[3], net.wb[0], net.wb[1], net.wb[2], net.wb[3],
                                                   net.w1g, net.wpair[1], net.wpair[2], net.w4ring,
                                                   net.kind == NET_FACE ? N_OUT_FACE_PAD : N_OUT_PAD);
  return cudaGetLastError();
}

cudaError_t acts_reserve(Acts& acts, long long cells, bool with_z) {
  if (acts.cells >= cells && (!with_z || acts.z[0])) return cudaSuccess;
  acts_free(acts);
  for (int l = 0; l < 3; ++l) {
    cudaError_t e = cudaMalloc(&acts.a[l], (size_t)cells * CG_HID * 16);
    if (e == cudaSuccess && with_z) e = cudaMalloc(&acts.z[l], (size_t)cells * CG_HID * 16);
    if (e != cudaSuccess) {
      acts_free(acts);
      return e;
    }
  }
  acts.cells = cells;
  return cudaSuccess;
}

void acts_free(Acts& acts) {
  for (int l = 0; l < 3; ++l) {
    cudaFree(acts.a[l]);
    cudaFree(acts.z[l]);
    acts.a[l] = nullptr;
    acts.z[l] = nullptr;
  }
  acts.cells = 0;
}

cudaError_t forward(const Net& net, const float* q, int B, int ny, int nx, Acts& acts, float* w,
                    float* raw, cudaStream_t s) {
  const ParamLayout L = param_layout();
  ConvArgs a{};
  a.nx = nx;
  a.ny = ny;
  a.plane = (long long)nx * ny;
  a.err = net.err;
  a.mean0 = net.mean[0];
  a.mean1 = net.mean[1];
  a.mean2 = net.mean[2];
  a.rstd0 = 1.f / net.std_[0];
  a.rstd1 = 1.f / net.std_[1];
  a.rstd2 = 1.f / net.std_[2];
  // layer 1: state -> a0
  a.q = q;
  a.wpk = net.wf[0];
  a.bias = net.params + L.b[0];
  a.y = acts.a[0];
  cudaError_t e = launch_conv<CG_IN0, HID, IN_STATE, OUT_RELU>(a, B, s);
  if (e != cudaSuccess) return e;
  // layers 2, 3
  for (int l = 1; l < 3; ++l) {
    a.x = acts.a[l - 1];
    a.wpk = net.wf[l];
    a.bias = net.params + L.b[l];
    a.y = acts.a[l];
    e = launch_conv<CG_HID, HID, IN_ACT, OUT_RELU>(a, B, s);
    if (e != cudaSuccess) return e;
  }
  // layer 4: a2 -> coefficients
  a.x = acts.a[2];
  a.wpk = net.wf[3];
  a.bias = net.params + L.b[3];
  if (raw) {
    a.w = raw;
    return launch_conv<CG_HID, N_OUT_PAD, IN_ACT, OUT_RAW>(a, B, s);
  }
  a.w = w;
  return launch_conv<CG_HID, N_OUT_PAD, IN_ACT, OUT_W>(a, B, s);
}

cudaError_t forward_faces(const Net& net, const float* q, int B, int ny, int nx, Acts& acts,
                          float* sides, float* raw, cudaStream_t s) {
  if (net.kind != NET_FACE) return cudaErrorInvalidValue;
  const ParamLayout L = param_layout(NET_FACE);
  ConvArgs a{};
  a.nx = nx;
  a.ny = ny;
  a.plane = (long long)nx * ny;
  a.err = net.err;
  a.mean0 = net.mean[0];
  a.mean1 = net.mean[1];
  a.mean2 = net.mean[2];
  a.rstd0 = 1.f / net.std_[0];
  a.rstd1 = 1.f / net.std_[1];
  a.rstd2 = 1.f / net.std_[2];
  a.std1 = net.std_[1];
  a.std2 = net.std_[2];
  // layer 1: state -> a0 (GeLU)
  a.q = q;
  a.wpk = net.wf[0];
  a.bias = net.params + L.b[0];
  a.y = acts.a[0];
  a.z = acts.z[0];
  cudaError_t e = launch_conv<CG_IN0, HID, IN_STATE, OUT_GELU>(a, B, s);
  if (e != cudaSuccess) return e;
  for (int l = 1; l < 3; ++l) {
    a.x = acts.a[l - 1];
    a.wpk = net.wf[l];
    a.bias = net.params + L.b[l];
    a.y = acts.a[l];
    a.z = acts.z[l];
    e = launch_conv<CG_HID, HID, IN_ACT, OUT_GELU>(a, B, s);
    if (e != cudaSuccess) return e;
  }
  a.z = nullptr;
  // layer 4: a2 -> the 12 side states
  a.x = acts.a[2];
  a.wpk = net.wf[3];
  a.bias = net.params + L.b[3];
  if (raw) {
    a.w = raw;
    return launch_conv<CG_HID, N_OUT_FACE_PAD, IN_ACT, OUT_SIDES_RAW>(a, B, s);
  }
  a.w = sides;
  return launch_conv<CG_HID, N_OUT_FACE_PAD, IN_ACT, OUT_SIDES>(a, B, s);
}

// ---------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------
namespace {

constexpr int DW_TILES = 16;         // 128-cell tiles per CTA of the weight-gradient kernel

// Cotangent of the normalised coefficients -> cotangent of the raw outputs
// (w = e + r - mean(r) per 3-tap stencil: dr_k = dw_k - mean(dw)), stored as
// BF16 in 6 channel groups (channels 36..47 zero).
__global__ void coeff_to_raw_kernel(const float* dw, uint16_t* dr, long long plane, long long cells) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= cells) return;
  const long long b = t / plane, cell = t - b * plane;
  const float* src = dw + b * N_OUT * plane + cell;
  float r[48];
#pragma unroll
  for (int s = 0; s < N_OUT / 3; ++s) {
    const float g0 = src[(3 * s) * plane], g1 = src[(3 * s + 1) * plane], g2 = src[(3 * s + 2) * plane];
    const float m = (g0 + g1 + g2) * (1.f / 3.f);
    r[3 * s] = g0 - m;
    r[3 * s + 1] = g1 - m;
    r[3 * s + 2] = g2 - m;
  }
#pragma unroll
  for (int k = N_OUT; k < 48; ++k) r[k] = 0.f;
#pragma unroll
  for (int g = 0; g < 6; ++g) {
    uint32_t pk[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) pk[j] = pack_bf16x2(r[8 * g + 2 * j], r[8 * g + 2 * j + 1]);
    *reinterpret_cast<uint4*>(dr + ((b * 6 + g) * plane + cell) * 8) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

// Cotangent of the side states -> cotangent of the raw outputs: Softplus'(r)
// = 1 - e^-h on the depths (h the side depth), std_v on the momenta; BF16
// in 2 channel groups (channels 12..15 zero).
__global__ void sides_to_raw_kernel(const float* ds, const float* sides, uint16_t* dr, long long plane,
                                    long long cells, float std1, float std2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= cells) return;
  const long long b = t / plane, cell = t - b * plane;
  const float* g = ds + b * N_OUT_FACE * plane + cell;
  const float* sd = sides + b * N_OUT_FACE * plane + cell;
  float r[16];
#pragma unroll
  for (int k = 0; k < N_OUT_FACE; ++k) {
    const int var = k % 3;
    const float f = var == 0 ? -expm1f(-sd[k * plane]) : (var == 1 ? std1 : std2);
    r[k] = g[k * plane] * f;
  }
#pragma unroll
  for (int k = N_OUT_FACE; k < 16; ++k) r[k] = 0.f;
#pragma unroll
  for (int gg = 0; gg < 2; ++gg) {
    uint32_t pk[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) pk[j] = pack_bf16x2(r[8 * gg + 2 * j], r[8 * gg + 2 * j + 1]);
    *reinterpret_cast<uint4*>(dr + ((b * 2 + gg) * plane + cell) * 8) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

// Weight and bias gradients of one layer as a deterministic reduction:
//   dW[co][ci][tap] = sum_cells dy[cell][co] * x[cell + off(tap)][ci],  db[co] = sum dy[cell][co].
// Each CTA handles DW_TILES tiles of 128 cells (staged like the forward:
// x in the tap-shifted position layout, FP32) and writes its partial sums;
// dw_reduce_kernel adds the partials in CTA order.  CI: input channels (3 for
// the first layer, read from the state and normalised), CO: output channels.
template <int CI, int CO, int CGO, bool ROW>
__global__ void __launch_bounds__(288) dw_partial_kernel(const uint16_t* x, const float* q,
                                                         const uint16_t* dy, float* part, int nx,
                                                         int ny, long long plane, long long ntiles,
                                                         float m0, float m1, float m2, float r0,
                                                         float r1, float r2) {
  constexpr int NP = npos_of<ROW>();
  extern __shared__ __align__(16) float dsm[];
  float* xs = dsm;                            // [NP][CI]
  float* ys = xs + NP * CI;                   // [TILE][CO]
  const int tid = threadIdx.x;
  constexpr bool rowmode = ROW;
  const int Lf = TILE + 2 * nx;
  const int npos = rowmode ? NPOS_ROW : 3 * Lf;
  constexpr int NE = 9 * CO;                  // (tap, co) pairs
  float acc[2][CI];
  float accb[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    accb[u] = 0.f;
#pragma unroll
    for (int c = 0; c < CI; ++c) acc[u][c] = 0.f;
  }
  const long long tiles_per_member = plane / TILE;
  for (int it = 0; it < DW_TILES; ++it) {
    const long long tile = (long long)blockIdx.x * DW_TILES + it;
    if (tile >= ntiles) break;
    const int b = (int)(tile / tiles_per_member);
    const int p0 = (int)(tile - (long long)b * tiles_per_member) * TILE;
    const int y0 = p0 / nx, x0 = p0 - (p0 / nx) * nx;
    __syncthreads();
    for (int n = tid; n < npos; n += blockDim.x) {
      int yy, xx;
      if (rowmode) {
        const int dyi = n / RW, xi = n - dyi * RW;
        yy = wrapi(y0 - 1 + dyi, ny);
        xx = wrapi(x0 - 1 + xi, nx);
      } else {
        const int dxi = n / Lf;
        const int c = p0 + (n - dxi * Lf) - nx;
        const int r = floordiv(c, nx);
        yy = wrapi(r, ny);
        xx = wrapi(c - r * nx + dxi - 1, nx);
      }
      const long long cell = (long long)yy * nx + xx;
      if constexpr (CI == 3) {
        const float* qb = q + (long long)b * 3 * plane;
        xs[n * 3 + 0] = __bfloat162float(__float2bfloat16_rn((qb[cell] - m0) * r0));
        xs[n * 3 + 1] = __bfloat162float(__float2bfloat16_rn((qb[plane + cell] - m1) * r1));
        xs[n * 3 + 2] = __bfloat162float(__float2bfloat16_rn((qb[2 * plane + cell] - m2) * r2));
      } else {
#pragma unroll
        for (int g = 0; g < CI / 8; ++g) {
          const uint4 v = *reinterpret_cast<const uint4*>(x + (((long long)b * (CI / 8) + g) * plane + cell) * 8);
          float* d = xs + n * CI + 8 * g;
          d[0] = bf16_lo(v.x); d[1] = bf16_hi(v.x); d[2] = bf16_lo(v.y); d[3] = bf16_hi(v.y);
          d[4] = bf16_lo(v.z); d[5] = bf16_hi(v.z); d[6] = bf16_lo(v.w); d[7] = bf16_hi(v.w);
        }
      }
    }
    for (int n = tid; n < TILE * CGO; n += blockDim.x) {
      const int m = n / CGO, g = n - (n / CGO) * CGO;
      const uint4 v = *reinterpret_cast<const uint4*>(dy + (((long long)b * CGO + g) * plane + p0 + m) * 8);
      const float vv[8] = {bf16_lo(v.x), bf16_hi(v.x), bf16_lo(v.y), bf16_hi(v.y),
                           bf16_lo(v.z), bf16_hi(v.z), bf16_lo(v.w), bf16_hi(v.w)};
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (8 * g + j < CO) ys[m * CO + 8 * g + j] = vv[j];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * 288;
      if (e >= NE) break;
      const int tap = e / CO, co = e - tap * CO;
      const int dy_ = tap / 3 - 1, dx_ = tap % 3 - 1;
      const int start = rowmode ? (1 + dy_) * RW + (1 + dx_) : (1 + dx_) * Lf + nx + dy_ * nx;
      for (int m = 0; m < TILE; ++m) {
        const float g = ys[m * CO + co];
        const float* xr = xs + (start + m) * CI;
#pragma unroll
        for (int c = 0; c < CI; ++c) acc[u][c] = fmaf(g, xr[c], acc[u][c]);
        accb[u] += g;
      }
    }
  }
  // partials: [cta][tap][co][ci] then [cta][9*CO*CI + co] for the bias
  float* pp = part + (long long)blockIdx.x * (NE * CI + CO);
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = tid + u * 288;
    if (e >= NE) break;
#pragma unroll
    for (int c = 0; c < CI; ++c) pp[e * CI + c] = acc[u][c];
    if (e < CO) pp[NE * CI + e] = accb[u];   // tap 0 threads carry the bias sums
  }
}

// Sum the partials in CTA order and add them to dparams (PyTorch layout).
template <int CI, int CO>
__global__ void dw_reduce_kernel(const float* part, int nparts, float* dW, float* db, float scale) {
  constexpr int NE = 9 * CO * CI;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NE + CO) return;
  float s = 0.f;
  for (int k = 0; k < nparts; ++k) s += part[(long long)k * (NE + CO) + i];
  if (i < NE) {
    const int c = i % CI, co = (i / CI) % CO, tap = i / (CI * CO);
    dW[(co * CI + c) * 9 + tap] += scale * s;
  } else {
    db[i - NE] += scale * s;
  }
}


// ---------------------------------------------------------------------------
// Weight and bias gradients on the tensor cores.
//
//   dW[co][ci][tap] = sum_p dy[p][co] x[p + off(tap)][ci],   db[co] = sum_p dy[p][co]
//
// as one GEMM per CTA over a contiguous range of cells p (K): D[r][co] =
// sum_p A[r][p] B[co][p] with A the 9-tap im2col of the layer input (rows
// r = tap * CI + ci) plus a row of ones (r = 9 CI, which yields db), and B
// the output cotangent (rows co, padded to NB).  Both operands are staged per
// K-tile of 64 cells in the K-major canonical layout (core matrices of 8
// rows x 8 cells, 16 bytes per row): the staging transposes the
// [group][cell][8 channels] records of global memory and applies the tap
// shifts with periodic wrap.  Two stage buffers alternate: the threads stage
// tile i+1 while the tensor core runs the MMAs of tile i (one thread issues
// MT x 4 tcgen05.mma of M = 128, N = NB, K = 16 per tile and commits them to
// the buffer's mbarrier).  The FP32 accumulators stay in TMEM for the CTA's
// whole range; the epilogue writes them as the CTA's partial sums, which
// dw_tc_reduce_kernel adds in CTA order (deterministic).  BF16 products are
// exact in FP32, so only the order of the FP32 sums differs from a CUDA-core
// reduction.
constexpr int DWK = 64;                  // cells per K-tile
constexpr int DW_CTAS = 304;             // CTAs (fixed: the partial sums do not depend on the GPU)
constexpr uint32_t DW_SBO = (DWK / 8) * 128;   // bytes between 8-row groups

template <int CI>
constexpr int dw_rows() { return 9 * CI + 1; }
template <int CI>
constexpr int dw_mt() { return (dw_rows<CI>() + 127) / 128; }
template <int CI, int NB>
constexpr int dw_buf_bytes() { return (dw_mt<CI>() * 128 + NB) * DWK * 2; }
template <int CI, int NB>
constexpr int dw_smem_bytes() { return 2 * dw_buf_bytes<CI, NB>() + 64; }

// Byte offset of element (row r, cell k) in a K-major tile of DWK cells.
__device__ __forceinline__ uint32_t dw_off(int r, int k) {
  return (uint32_t)(r >> 3) * DW_SBO + (uint32_t)(k >> 3) * 128u + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// Periodic neighbour of cell p (row-major nx x ny plane) at offset (dy, dx),
// dy, dx in {-1, 0, 1}.
__device__ __forceinline__ long long shifted_cell(int p, int nx, int ny, int dy, int dx, int lg) {
  const int y = lg >= 0 ? p >> lg : p / nx, x = p - y * nx;
  int ys = y + dy, xs = x + dx;
  ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
  xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
  return (long long)ys * nx + xs;
}

template <int CI, int CO, int CGO>
__global__ void __launch_bounds__(NT) dw_tc_kernel(const uint16_t* x, const float* q, const uint16_t* dy,
                                                   float* part, int nx, int ny, long long plane,
                                                   long long ntiles, float m0, float m1, float m2, float r0,
                                                   float r1, float r2, unsigned* err) {
  constexpr int NB = 8 * CGO;            // padded output channels (N)
  constexpr int MT = dw_mt<CI>();
  constexpr int ROWS = MT * 128;
  constexpr int BUF = dw_buf_bytes<CI, NB>();
  static_assert(NB % 16 == 0 && NB <= 256, "N of the MMA");
  static_assert(MT * NB <= 256, "TMEM columns");
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * BUF);   // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x;
  const long long t0 = (long long)blockIdx.x * ntiles / gridDim.x;
  const long long t1 = (long long)(blockIdx.x + 1) * ntiles / gridDim.x;
  const long long tiles_per_member = plane / DWK;

  // constant rows of both buffers: the ones row (bias) and the zero padding
  for (int buf = 0; buf < 2; ++buf) {
    uint8_t* A = smem + buf * BUF;
    for (int i = tid; i < (ROWS - 9 * CI) * DWK; i += NT) {
      const int r = 9 * CI + i / DWK, k = i % DWK;
      *reinterpret_cast<uint16_t*>(A + dw_off(r, k)) = r == 9 * CI ? (uint16_t)0x3F80u : (uint16_t)0u;
    }
    uint8_t* Bm = A + ROWS * DWK * 2;
    for (int i = tid; i < (NB - CO) * DWK; i += NT) {
      const int n = CO + i / DWK, k = i % DWK;
      *reinterpret_cast<uint16_t*>(Bm + dw_off(n, k)) = 0;
    }
  }
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if ((tid >> 5) == 0) tc::tmem_alloc(tslot, 256);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NB);
  const int lg = (nx & (nx - 1)) == 0 ? __ffs(nx) - 1 : -1;   // power-of-two width: shift
  bool ok = true;
  int issued = 0;                        // tiles whose MMAs were issued (the same in every thread)

  for (long long tile = t0; tile < t1; ++tile) {
    const int i = (int)(tile - t0);
    const int buf = i & 1;
    uint8_t* A = smem + buf * BUF;
    uint8_t* Bm = A + ROWS * DWK * 2;
    // the buffer is free once the MMAs of tile i - 2 are done
    if (i >= 2) {
      const bool w = tc::mbar_wait_bounded(&mbar[buf], (uint32_t)((i - 2) >> 1) & 1u, WAIT_ITERS);
      ok = __syncthreads_and(w) && ok;
      if (!ok) break;
    }
    const int b = (int)(tile / tiles_per_member);
    const int p0 = (int)(tile - (long long)b * tiles_per_member) * DWK;
    // B: output cotangent, one 16-byte record (8 channels of one cell) per item
    for (int it = tid; it < DWK * CGO; it += NT) {
      const int k = it % DWK, g = it / DWK;
      const uint4 v = *reinterpret_cast<const uint4*>(dy + (((long long)b * CGO + g) * plane + p0 + k) * 8);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = 8 * g + j;
        if (n < NB)
          *reinterpret_cast<uint16_t*>(Bm + dw_off(n, k)) = (uint16_t)(w4[j >> 1] >> (16 * (j & 1)));
      }
    }
    // A: the input at the 9 tap-shifted cells (periodic), rows tap * CI + ci
    for (int it = tid; it < DWK * 9; it += NT) {
      const int k = it % DWK, tap = it / DWK;
      const long long cell = shifted_cell(p0 + k, nx, ny, tap / 3 - 1, tap % 3 - 1, lg);
      if constexpr (CI == 3) {
        const float* qb = q + (long long)b * 3 * plane;
        const float v[3] = {(qb[cell] - m0) * r0, (qb[plane + cell] - m1) * r1, (qb[2 * plane + cell] - m2) * r2};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const __nv_bfloat16 h = __float2bfloat16_rn(v[c]);
          *reinterpret_cast<__nv_bfloat16*>(A + dw_off(tap * 3 + c, k)) = h;
        }
      } else {
#pragma unroll
        for (int g = 0; g < CI / 8; ++g) {
          const uint4 v = *reinterpret_cast<const uint4*>(x + (((long long)b * (CI / 8) + g) * plane + cell) * 8);
          const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int j = 0; j < 8; ++j)
            *reinterpret_cast<uint16_t*>(A + dw_off(tap * CI + 8 * g + j, k)) =
                (uint16_t)(w4[j >> 1] >> (16 * (j & 1)));
        }
      }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(Bm);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
        for (int ks = 0; ks < DWK / 16; ++ks) {
          const uint64_t ad = tc::sdesc(a0 + mt * 16 * DW_SBO + ks * 256, 128, DW_SBO);
          const uint64_t bd = tc::sdesc(b0 + ks * 256, 128, DW_SBO);
          tc::mma_bf16(tmem + mt * NB, ad, bd, idesc, i > 0 || ks > 0);
        }
      }
      tc::mma_commit(&mbar[buf]);
    }
    issued = i + 1;
  }
  // every commit issued must have landed before TMEM is read or released: the
  // last tile issued on each buffer (bounded waits; after a timeout the CTA
  // flags the error and still releases its TMEM)
  for (int bb = 0; bb < 2; ++bb) {
    const int last = issued - 1 - ((issued - 1 - bb) & 1);   // largest tile < issued on buffer bb
    if (last >= 0) {
      const bool w = tc::mbar_wait_bounded(&mbar[bb], (uint32_t)(last >> 1) & 1u, WAIT_ITERS);
      ok = __syncthreads_and(w) && ok;
    }
  }
  const int n = issued;
  tc::fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicOr(err, 1u);
  } else {
    // warp w holds TMEM lanes 32w .. 32w+31 = rows 128 mt + 32 w + lane
    const int warp = tid >> 5, lane = tid & 31;
    float* pp = part + (long long)blockIdx.x * ROWS * CO;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int r = mt * 128 + warp * 32 + lane;
#pragma unroll
      for (int c0 = 0; c0 < NB; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + mt * NB + c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < CO) pp[(long long)(c0 + j) * ROWS + r] = n > 0 ? v[j] : 0.f;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if ((tid >> 5) == 0) tc::tmem_dealloc(tmem, 256);
}

// Sum the CTAs' partial sums into dparams (PyTorch layout).  A CTA's
// partials are [CO][ROWS] (column co of the accumulator, row r = tap * CI +
// ci gives dW[co][ci][tap], row 9 CI gives db; the lanes of a warp write
// consecutive rows).  A block of 8 warps handles 32 consecutive (co, r)
// outputs; warp w sums partials [w P / 8, (w+1) P / 8) in order, then the 8
// sums are added in warp order (a fixed order: the result does not depend
// on timing).
template <int CI, int CO, int CIP = CI>
__global__ void __launch_bounds__(256) dw_tc_reduce_kernel(const float* part, int nparts, float* dW, float* db,
                                                           float scale) {
  // CIP: input channels of the GEMM rows (CI padded; rows of channels >= CI are dropped)
  constexpr int ROWS = dw_mt<CIP>() * 128;
  constexpr int NR = 9 * CIP + 1;
  constexpr int NE = NR * CO;
  __shared__ float sh[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 32 + lane;
  const int co = i / NR, r = i - co * NR;
  float s = 0.f;
  if (i < NE) {
    const int k0 = warp * nparts / 8, k1 = (warp + 1) * nparts / 8;
    const float* src = part + co * ROWS + r;
    int k = k0;
    // eight loads in flight, then added in order (the same sum as one by one)
    for (; k + 8 <= k1; k += 8) {
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = src[(long long)(k + j) * ROWS * CO];
#pragma unroll
      for (int j = 0; j < 8; ++j) s += v[j];
    }
    for (; k < k1; ++k) s += src[(long long)k * ROWS * CO];
  }
  sh[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && i < NE) {
    float t = sh[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) t += sh[w][lane];
    if (r < 9 * CIP) {
      const int tap = r / CIP, c = r - tap * CIP;
      if (c < CI) dW[(co * CI + c) * 9 + tap] += scale * t;
    } else {
      db[co] += scale * t;
    }
  }
}

// The same GEMM with the staging done by the copy engines and the matrix
// instructions (CI a multiple of 8): the raw 16-byte records the tile needs
// (the input at the three rows or x-shifted strips of positions the tile's
// taps read, and the cotangent of the tile's cells) arrive by cp.async, two
// tiles ahead of use (two raw buffers); every warp then transposes 8x8 blocks
// (8 cells x 8 channels) with ldmatrix.trans and writes them as K-major rows
// with stmatrix.  The shared-memory addresses of a warp's blocks do not
// depend on the tile and are computed once.
__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t row_addr, uint32_t (&w)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "r"(row_addr));
}
__device__ __forceinline__ void stmatrix_x4(uint32_t row_addr, const uint32_t (&w)[4]) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1, %2, %3, %4};\n"
               :: "r"(row_addr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]) : "memory");
}

// Raw positions of a 64-cell tile: row mode (nx a multiple of DWK) 3 rows of
// DWK + 2 cells; strip mode (nx < DWK dividing it) 3 x-shifted strips of
// DWK + 2 nx cells.
constexpr int DWT = 256;                 // threads of the cp.async/ldmatrix weight-gradient kernel
constexpr int DW_RW = DWK + 2;
constexpr int DW_NPOS_ROW = 3 * DW_RW;
constexpr int DW_NPOS_FLAT = 3 * (DWK + 2 * (DWK / 2));
template <bool ROW>
constexpr int dw_npos() { return ROW ? DW_NPOS_ROW : DW_NPOS_FLAT; }
template <int CI, int CGO, bool ROW>
constexpr int dwx_raw_bytes() { return (CI / 8) * dw_npos<ROW>() * 16 + CGO * DWK * 16; }
template <int CI, int CGO, bool ROW>
constexpr int dwx_smem_bytes() {
  return 2 * dwx_raw_bytes<CI, CGO, ROW>() + (dw_mt<CI>() * 128 + 8 * CGO) * DWK * 2 + 64;
}

template <int CI, int CO, int CGO, bool ROW>
__global__ void __launch_bounds__(DWT) dw_tx_kernel(const uint16_t* x, const uint16_t* dy, float* part, int nx,
                                                   int ny, long long plane, long long ntiles, unsigned* err) {
  constexpr int CG = CI / 8;
  constexpr int NB = 8 * CGO;
  constexpr int MT = dw_mt<CI>();
  constexpr int ROWS = MT * 128;
  constexpr int NP = dw_npos<ROW>();
  constexpr int RAW = dwx_raw_bytes<CI, CGO, ROW>();
  constexpr int NW = DWT / 32;
  constexpr int A_X4 = 9 * CG * 8 / 4, B_X4 = CGO * 8 / 4;   // ldmatrix.x4 blocks of A, B per tile
  constexpr int A_PER_WARP = (A_X4 + NW - 1) / NW, B_PER_WARP = (B_X4 + NW - 1) / NW;
  static_assert(CI % 8 == 0 && NB % 16 == 0 && MT * NB <= 256, "shape of the MMA and TMEM columns");
  constexpr uint32_t NCOLS = MT * NB <= 32 ? 32u : (MT * NB <= 64 ? 64u : (MT * NB <= 128 ? 128u : 256u));
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* R = smem;                                   // 2 x {[CG][NP][16 B] input, [CGO][DWK][16 B] cotangent}
  uint8_t* A = smem + 2 * RAW;                         // K-major [ROWS][DWK]
  uint8_t* Bm = A + ROWS * DWK * 2;                    // K-major [NB][DWK]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Bm + NB * DWK * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long t0 = (long long)blockIdx.x * ntiles / gridDim.x;
  const long long t1 = (long long)(blockIdx.x + 1) * ntiles / gridDim.x;
  const long long tiles_per_member = plane / DWK;
  const int lg = (nx & (nx - 1)) == 0 ? __ffs(nx) - 1 : -1;
  const int Lf = DWK + 2 * nx;                         // strip mode

  // the ones row (bias) and the zero padding of A, once
  for (int i = tid; i < (ROWS - 9 * CI) * DWK; i += DWT) {
    const int r = 9 * CI + i / DWK, k = i % DWK;
    *reinterpret_cast<uint16_t*>(A + dw_off(r, k)) = r == 9 * CI ? (uint16_t)0x3F80u : (uint16_t)0u;
  }
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tslot, NCOLS);

  // this lane's row addresses of its warp's 8x8 blocks: block t = (tap, g,
  // kb) of A reads raw positions start(tap) + 8 kb .. + 7 of group g and
  // writes rows tap CI + 8 g .. + 7 at cells 8 kb .. + 7; block (g, kb) of B
  // likewise from the cotangent
  const uint32_t r_base = tc::smem_u32(R), a_base = tc::smem_u32(A), b_base = tc::smem_u32(Bm);
  uint32_t a_ld[A_PER_WARP], a_st[A_PER_WARP], b_ld[B_PER_WARP], b_st[B_PER_WARP];
  {
    const int m = lane >> 3, row = lane & 7;
#pragma unroll
    for (int k = 0; k < A_PER_WARP; ++k) {
      const int ins = warp + NW * k < A_X4 ? warp + NW * k : 0;   // (a warp past the end skips it)
      const int t = 4 * ins + m, kb = t & 7, g = (t >> 3) % CG, tap = (t >> 3) / CG;
      const int dy_ = tap / 3 - 1, dx_ = tap % 3 - 1;
      const int start = ROW ? (1 + dy_) * DW_RW + (1 + dx_) : (1 + dx_) * Lf + nx + dy_ * nx;
      a_ld[k] = (uint32_t)((g * NP + start + 8 * kb + row) * 16);
      a_st[k] = a_base + dw_off(tap * CI + 8 * g + row, 8 * kb);
    }
#pragma unroll
    for (int k = 0; k < B_PER_WARP; ++k) {
      const int ins = warp + NW * k < B_X4 ? warp + NW * k : 0;
      const int t = 4 * ins + m, kb = t & 7, g = t >> 3;
      b_ld[k] = (uint32_t)(CG * NP * 16 + (g * DWK + 8 * kb + row) * 16);
      b_st[k] = b_base + dw_off(8 * g + row, 8 * kb);
    }
  }

  // raw records of tile `tile` into raw buffer `buf` (cp.async; the caller commits)
  auto stage_raw = [&](long long tile, int buf) {
    uint8_t* Rb = R + buf * RAW;
    uint8_t* RBb = Rb + CG * NP * 16;
    const int b = (int)(tile / tiles_per_member);
    const int p0 = (int)(tile - (long long)b * tiles_per_member) * DWK;
    const int y0 = lg >= 0 ? p0 >> lg : p0 / nx, x0 = p0 - y0 * nx;
    const int npos = ROW ? DW_NPOS_ROW : 3 * Lf;
    for (int n = tid; n < npos; n += DWT) {
      int yy, xx;
      if (ROW) {
        const int dyi = (n >= DW_RW) + (n >= 2 * DW_RW), xi = n - dyi * DW_RW;
        yy = wrap1(y0 - 1 + dyi, ny);
        xx = wrap1(x0 - 1 + xi, nx);
      } else {
        const int dxi = (n >= Lf) + (n >= 2 * Lf);
        const int c = p0 + (n - dxi * Lf) - nx;
        const int r = lg >= 0 ? (c >> lg) : floordiv(c, nx);
        yy = wrap1(r, ny);
        xx = wrap1(c - r * nx + dxi - 1, nx);
      }
      const long long cell = (long long)yy * nx + xx;
#pragma unroll
      for (int g = 0; g < CG; ++g)
        cp_async16(Rb + (g * NP + n) * 16, x + (((long long)b * CG + g) * plane + cell) * 8);
    }
    for (int n = tid; n < CGO * DWK; n += DWT) {
      const int g = n / DWK, k = n - g * DWK;
      cp_async16(RBb + n * 16, dy + (((long long)b * CGO + g) * plane + p0 + k) * 8);
    }
  };

  if (t0 < t1) stage_raw(t0, 0);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  if (t0 + 1 < t1) stage_raw(t0 + 1, 1);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NB);
  bool ok = true;
  int issued = 0;
  for (long long tile = t0; tile < t1; ++tile) {
    const int i = (int)(tile - t0);
    const uint32_t rb = r_base + (uint32_t)((i & 1) * RAW);
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // this tile's records (one later group may pend)
    // A and B are free once the MMAs of the previous tile are done
    bool w = true;
    if (i >= 1) w = tc::mbar_wait_bounded(mbar, (uint32_t)(i - 1) & 1u, WAIT_ITERS);
    ok = __syncthreads_and(w) && ok;
    if (!ok) break;
    tc::fence_after_sync();
    // all of this warp's loads first, then the stores (the matrix
    // instructions are not reordered across each other)
    {
      uint32_t va[A_PER_WARP][4], vb[B_PER_WARP][4];
#pragma unroll
      for (int k = 0; k < A_PER_WARP; ++k)
        if (A_X4 % NW == 0 || warp + NW * k < A_X4) ldmatrix_x4_trans(rb + a_ld[k], va[k]);
#pragma unroll
      for (int k = 0; k < B_PER_WARP; ++k)
        if (B_X4 % NW == 0 || warp + NW * k < B_X4) ldmatrix_x4_trans(rb + b_ld[k], vb[k]);
#pragma unroll
      for (int k = 0; k < A_PER_WARP; ++k)
        if (A_X4 % NW == 0 || warp + NW * k < A_X4) stmatrix_x4(a_st[k], va[k]);
#pragma unroll
      for (int k = 0; k < B_PER_WARP; ++k)
        if (B_X4 % NW == 0 || warp + NW * k < B_X4) stmatrix_x4(b_st[k], vb[k]);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
        for (int ks = 0; ks < DWK / 16; ++ks) {
          const uint64_t ad = tc::sdesc(a_base + mt * 16 * DW_SBO + ks * 256, 128, DW_SBO);
          const uint64_t bd = tc::sdesc(b_base + ks * 256, 128, DW_SBO);
          tc::mma_bf16(tmem + mt * NB, ad, bd, idesc, i > 0 || ks > 0);
        }
      }
      tc::mma_commit(mbar);
    }
    issued = i + 1;
    // this raw buffer is read: the records of tile + 2 go into it
    if (tile + 2 < t1) stage_raw(tile + 2, i & 1);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  if (issued > 0) {
    const bool w = tc::mbar_wait_bounded(mbar, (uint32_t)(issued - 1) & 1u, WAIT_ITERS);
    ok = __syncthreads_and(w) && ok;
  }
  tc::fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicOr(err, 1u);
  } else {
    // warp w reads TMEM lanes 32 (w % 4) ..; warps w and w + 4 take
    // alternate 16-column chunks
    float* pp = part + (long long)blockIdx.x * ROWS * CO;
    const int lq = warp & 3, half = warp >> 2;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int r = mt * 128 + lq * 32 + lane;
#pragma unroll
      for (int c0 = 0; c0 < NB; c0 += 16) {
        if (((c0 >> 4) & 1) != half) continue;
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + mt * NB + c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < CO) pp[(long long)(c0 + j) * ROWS + r] = issued > 0 ? v[j] : 0.f;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, NCOLS);
}

template <int CI, int CO, int CGO, bool ROW>
cudaError_t launch_dw_tx(const uint16_t* x, const uint16_t* dy, float* part, int nx, int ny, long long plane,
                         long long ntiles, int nctas, const Net& net, cudaStream_t s) {
  constexpr int smem = dwx_smem_bytes<CI, CGO, ROW>();
  auto kern = dw_tx_kernel<CI, CO, CGO, ROW>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  kern<<<nctas, DWT, smem, s>>>(x, dy, part, nx, ny, plane, ntiles, net.err);
  return cudaGetLastError();
}

// Where a weight gradient's partial-sum reduction runs: by default on the
// stream of its partial-sum kernel; with rs set, on rs after that kernel
// (event ev), so that the stream goes on with the next kernel.
struct RedOn {
  cudaStream_t rs = nullptr;
  cudaEvent_t ev = nullptr;
};
inline cudaError_t red_stream(cudaStream_t s, const RedOn& r, cudaStream_t& out) {
  out = s;
  if (!r.rs) return cudaSuccess;
  cudaError_t e = cudaEventRecord(r.ev, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(r.rs, r.ev, 0);
  out = r.rs;
  return e;
}

template <int CI, int CO, int CGO>
cudaError_t weight_grad_tc(const uint16_t* x, const float* q, const uint16_t* dy, float* dW, float* db,
                           float* part, int B, int ny, int nx, const Net& net, float scale, cudaStream_t s,
                           const RedOn& ro) {
  cudaStream_t rs = s;
  const long long plane = (long long)nx * ny;
  const long long ntiles = (long long)B * (plane / DWK);
  const int nctas = (int)(ntiles < DW_CTAS ? ntiles : DW_CTAS);
  if constexpr (CI % 8 == 0) {
    // staging by cp.async + ldmatrix / stmatrix: a tile lies within one row
    // (nx a multiple of 64) or covers whole rows (nx dividing 64)
    if (nx % DWK == 0 || DWK % nx == 0) {
      cudaError_t e;
      if (nx % DWK == 0) e = launch_dw_tx<CI, CO, CGO, true>(x, dy, part, nx, ny, plane, ntiles, nctas, net, s);
      else e = launch_dw_tx<CI, CO, CGO, false>(x, dy, part, nx, ny, plane, ntiles, nctas, net, s);
      if (e != cudaSuccess) return e;
      if ((e = red_stream(s, ro, rs)) != cudaSuccess) return e;
      const int ne = (9 * CI + 1) * CO;
      dw_tc_reduce_kernel<CI, CO><<<(ne + 31) / 32, 256, 0, rs>>>(part, nctas, dW, db, scale);
      return cudaGetLastError();
    }
  }
  constexpr int smem = dw_smem_bytes<CI, 8 * CGO>();
  auto kern = dw_tc_kernel<CI, CO, CGO>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  kern<<<nctas, NT, smem, s>>>(x, q, dy, part, nx, ny, plane, ntiles, net.mean[0], net.mean[1], net.mean[2],
                               1.f / net.std_[0], 1.f / net.std_[1], 1.f / net.std_[2], net.err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = red_stream(s, ro, rs)) != cudaSuccess) return e;
  const int ne = (9 * CI + 1) * CO;
  dw_tc_reduce_kernel<CI, CO><<<(ne + 31) / 32, 256, 0, rs>>>(part, nctas, dW, db, scale);
  return cudaGetLastError();
}

template <int CI, int CO, int CGO, bool ROW>
cudaError_t weight_grad_t(const uint16_t* x, const float* q, const uint16_t* dy, float* dW, float* db,
                          float* part, int B, int ny, int nx, const Net& net, float scale,
                          cudaStream_t s, const RedOn& ro) {
  const long long plane = (long long)nx * ny;
  const long long ntiles = (long long)B * (plane / TILE);
  const int nctas = (int)((ntiles + DW_TILES - 1) / DW_TILES);
  const int smem = (npos_of<ROW>() * CI + TILE * CO) * 4;
  auto kern = dw_partial_kernel<CI, CO, CGO, ROW>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  kern<<<nctas, 288, smem, s>>>(x, q, dy, part, nx, ny, plane, ntiles, net.mean[0], net.mean[1],
                                net.mean[2], 1.f / net.std_[0], 1.f / net.std_[1], 1.f / net.std_[2]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cudaStream_t rs = s;
  if ((e = red_stream(s, ro, rs)) != cudaSuccess) return e;
  const int ne = 9 * CO * CI + CO;
  dw_reduce_kernel<CI, CO><<<(ne + 255) / 256, 256, 0, rs>>>(part, nctas, dW, db, scale);
  return cudaGetLastError();
}

template <int CI, int CO, int CGO>
cudaError_t weight_grad(const uint16_t* x, const float* q, const uint16_t* dy, float* dW, float* db,
                        float* part, int B, int ny, int nx, const Net& net, float scale,
                        cudaStream_t s, const RedOn& ro = RedOn{}) {
  if (((long long)nx * ny) % DWK == 0)
    return weight_grad_tc<CI, CO, CGO>(x, q, dy, dW, db, part, B, ny, nx, net, scale, s, ro);
  if (nx % TILE == 0)
    return weight_grad_t<CI, CO, CGO, true>(x, q, dy, dW, db, part, B, ny, nx, net, scale, s, ro);
  return weight_grad_t<CI, CO, CGO, false>(x, q, dy, dW, db, part, B, ny, nx, net, scale, s, ro);
}

// The normalised state as the first layer's BF16 input records [B][1][plane][8]
// (channels h, hu, hv, then zeros), rounded as the forward convolution rounds it.
__global__ void pack_input_kernel(const float* q, uint16_t* x0, long long plane, long long cells, float m0,
                                  float m1, float m2, float r0, float r1, float r2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= cells) return;
  const long long b = t / plane, cell = t - b * plane;
  const float* qb = q + b * 3 * plane + cell;
  const float h0 = (qb[0] - m0) * r0, h1 = (qb[plane] - m1) * r1, h2 = (qb[2 * plane] - m2) * r2;
  *reinterpret_cast<uint4*>(x0 + t * 8) = make_uint4(pack_bf16x2(h0, h1), pack_bf16x2(h2, 0.f), 0u, 0u);
}

// Backward of the first layer (input: the normalised state, 3 channels): dW1
// and db1 from the layer's output cotangent da0, and dq += dX / std.  dW runs
// on the tensor cores over the state packed as 8-channel BF16 records (in
// g.dr, free at this point), its rows of the 5 zero channels dropped in the
// reduction; dX is the convolution with the flipped weights (N = 16).  dW
// goes to stream sw, dX to s; both only read da0.
cudaError_t backward_first(const Net& net, const float* q, const uint16_t* da0, const ParamLayout& L, int B,
                           int ny, int nx, Grads& g, float* part, float* dq, float* dparams, float scale,
                           cudaStream_t sw, cudaStream_t s, const RedOn& ro) {
  const long long plane = (long long)nx * ny, cells = (long long)B * plane;
  cudaError_t e;
  if (plane % DWK == 0 && (nx % DWK == 0 || DWK % nx == 0)) {
    pack_input_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, sw>>>(
        q, g.dr, plane, cells, net.mean[0], net.mean[1], net.mean[2], 1.f / net.std_[0], 1.f / net.std_[1],
        1.f / net.std_[2]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long ntiles = (long long)B * (plane / DWK);
    const int nctas = (int)(ntiles < DW_CTAS ? ntiles : DW_CTAS);
    if (nx % DWK == 0) e = launch_dw_tx<8, HID, 4, true>(g.dr, da0, part, nx, ny, plane, ntiles, nctas, net, sw);
    else e = launch_dw_tx<8, HID, 4, false>(g.dr, da0, part, nx, ny, plane, ntiles, nctas, net, sw);
    if (e != cudaSuccess) return e;
    cudaStream_t rs = sw;
    if ((e = red_stream(sw, ro, rs)) != cudaSuccess) return e;
    constexpr int ne = (9 * 8 + 1) * HID;
    dw_tc_reduce_kernel<3, HID, 8><<<(ne + 31) / 32, 256, 0, rs>>>(part, nctas, dparams + L.w[0],
                                                                   dparams + L.b[0], scale);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    if ((e = weight_grad<3, HID, 4>(nullptr, q, da0, dparams + L.w[0], dparams + L.b[0], part, B, ny, nx, net,
                                    scale, sw, ro)) != cudaSuccess)
      return e;
  }
  if (dq) {
    ConvArgs a{};
    a.nx = nx;
    a.ny = ny;
    a.plane = plane;
    a.err = net.err;
    a.x = da0;
    a.wpk = net.wb[0];
    a.w = dq;
    a.rstd0 = 1.f / net.std_[0];
    a.rstd1 = 1.f / net.std_[1];
    a.rstd2 = 1.f / net.std_[2];
    if ((e = launch_conv<CG_HID, DQ_N, IN_ACT, OUT_DQ>(a, B, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

long long backward_partials_floats(int B, int ny, int nx) {
  const long long ntiles = (long long)B * ((long long)nx * ny / TILE);
  const long long nctas = (ntiles + DW_TILES - 1) / DW_TILES;
  const long long cuda_cores = nctas * (9 * N_OUT * HID + N_OUT);
  const long long tensor = (long long)DW_CTAS * dw_mt<HID>() * 128 * N_OUT;   // largest tensor-core layer
  return cuda_cores > tensor ? cuda_cores : tensor;
}

cudaError_t backward_reserve(Grads& g, long long cells, long long partial_floats) {
  if (!g.aux) {
    cudaError_t e = cudaStreamCreateWithFlags(&g.aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.red, cudaStreamNonBlocking);
    for (int i = 0; i < Grads::NEV && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&g.ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  if (g.cells < cells) {
    cudaFree(g.dr);
    cudaFree(g.da[0]);
    cudaFree(g.da[1]);
    g.dr = nullptr;
    g.da[0] = g.da[1] = nullptr;
    g.cells = 0;
    cudaError_t e = cudaMalloc(&g.dr, (size_t)cells * 6 * 16);
    if (e == cudaSuccess) e = cudaMalloc(&g.da[0], (size_t)cells * CG_HID * 16);
    if (e == cudaSuccess) e = cudaMalloc(&g.da[1], (size_t)cells * CG_HID * 16);
    if (e != cudaSuccess) return e;
    g.cells = cells;
  }
  if (g.part_floats < partial_floats) {
    cudaFree(g.part);
    cudaFree(g.part2);
    g.part = g.part2 = nullptr;
    g.part_floats = 0;
    cudaError_t e = cudaMalloc(&g.part, sizeof(float) * partial_floats);
    if (e == cudaSuccess) e = cudaMalloc(&g.part2, sizeof(float) * partial_floats);
    if (e != cudaSuccess) return e;
    g.part_floats = partial_floats;
  }
  return cudaSuccess;
}

void backward_free(Grads& g) {
  if (g.aux) cudaStreamSynchronize(g.aux);
  if (g.red) cudaStreamSynchronize(g.red);
  cudaFree(g.dr);
  cudaFree(g.da[0]);
  cudaFree(g.da[1]);
  cudaFree(g.part);
  cudaFree(g.part2);
  for (int i = 0; i < Grads::NEV; ++i)
    if (g.ev[i]) cudaEventDestroy(g.ev[i]);
  if (g.aux) cudaStreamDestroy(g.aux);
  if (g.red) cudaStreamDestroy(g.red);
  g = Grads{};
}

namespace {
// `to` waits for the work enqueued so far on `from` (event slot i).
cudaError_t stream_after(Grads& g, int i, cudaStream_t from, cudaStream_t to) {
  cudaError_t e = cudaEventRecord(g.ev[i], from);
  return e == cudaSuccess ? cudaStreamWaitEvent(to, g.ev[i], 0) : e;
}
}  // namespace

cudaError_t backward(const Net& net, const float* q, int B, int ny, int nx, const Acts& acts,
                     const float* dw, float* dq, float* dparams, float scale, Grads& g,
                     cudaStream_t s) {
  const long long cells = (long long)B * nx * ny;
  coeff_to_raw_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(dw, g.dr, (long long)nx * ny, cells);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return backward_from_raw(net, q, B, ny, nx, acts, dq, dparams, scale, g, s);
}

cudaError_t backward_from_raw(const Net& net, const float* q, int B, int ny, int nx, const Acts& acts,
                              float* dq, float* dparams, float scale, Grads& g, cudaStream_t s) {
  const ParamLayout L = param_layout();
  const long long plane = (long long)nx * ny;
  cudaError_t e;

  // Each layer's dW (stream g.aux, in layer order) runs beside its dX
  // (stream s): both only read the layer's output cotangent.  dX of layer 2
  // overwrites da[0], which dW3 reads: it waits.
  cudaStream_t w = g.aux;
  ConvArgs a{};
  a.nx = nx;
  a.ny = ny;
  a.plane = plane;
  a.err = net.err;
  // (the reductions of an earlier call were joined into s: its buffers are
  // free, which the two buffer events restate from s, so that every wait
  // below refers to work of this call, as a graph capture requires)
  if ((e = cudaEventRecord(g.ev[6], s)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(g.ev[7], s)) != cudaSuccess) return e;
  if ((e = stream_after(g, 0, s, w)) != cudaSuccess) return e;
  // the reductions run on g.red; layers alternate between two partial
  // buffers, and a layer's partial sums wait for the reduction that last
  // read its buffer
  const RedOn ro{g.red, g.ev[8]};
  float* part[2] = {g.part, g.part2};
  // layer 4: dW4, db4 from (dr, a3); dX -> da[0] masked by a3
  if ((e = cudaStreamWaitEvent(w, g.ev[6], 0)) != cudaSuccess) return e;
  if ((e = weight_grad<HID, N_OUT, 6>(acts.a[2], nullptr, g.dr, dparams + L.w[3], dparams + L.b[3],
                                      part[0], B, ny, nx, net, scale, w, ro)) != cudaSuccess)
    return e;
  if ((e = cudaEventRecord(g.ev[6], g.red)) != cudaSuccess) return e;
  a.x = g.dr;
  a.wpk = net.wb[3];
  a.mask = acts.a[2];
  a.y = g.da[0];
  if ((e = launch_conv<6, HID, IN_ACT, OUT_MASK>(a, B, s)) != cudaSuccess) return e;
  if ((e = stream_after(g, 1, s, w)) != cudaSuccess) return e;
  // layer 3: dW3 from (da0, a2); dX -> da[1] masked by a2
  if ((e = cudaStreamWaitEvent(w, g.ev[7], 0)) != cudaSuccess) return e;
  if ((e = weight_grad<HID, HID, 4>(acts.a[1], nullptr, g.da[0], dparams + L.w[2], dparams + L.b[2],
                                    part[1], B, ny, nx, net, scale, w, ro)) != cudaSuccess)
    return e;
  if ((e = cudaEventRecord(g.ev[7], g.red)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(g.ev[2], w)) != cudaSuccess) return e;   // dW3 has read da[0]
  a.x = g.da[0];
  a.wpk = net.wb[2];
  a.mask = acts.a[1];
  a.y = g.da[1];
  if ((e = launch_conv<CG_HID, HID, IN_ACT, OUT_MASK>(a, B, s)) != cudaSuccess) return e;
  if ((e = stream_after(g, 3, s, w)) != cudaSuccess) return e;
  // layer 2: dW2 from (da1, a1); dX -> da[0] masked by a1
  if ((e = cudaStreamWaitEvent(w, g.ev[6], 0)) != cudaSuccess) return e;
  if ((e = weight_grad<HID, HID, 4>(acts.a[0], nullptr, g.da[1], dparams + L.w[1], dparams + L.b[1],
                                    part[0], B, ny, nx, net, scale, w, ro)) != cudaSuccess)
    return e;
  if ((e = cudaEventRecord(g.ev[6], g.red)) != cudaSuccess) return e;
  a.x = g.da[1];
  a.wpk = net.wb[1];
  a.mask = acts.a[0];
  a.y = g.da[0];
  if ((e = cudaStreamWaitEvent(s, g.ev[2], 0)) != cudaSuccess) return e;
  if ((e = launch_conv<CG_HID, HID, IN_ACT, OUT_MASK>(a, B, s)) != cudaSuccess) return e;
  if ((e = stream_after(g, 4, s, w)) != cudaSuccess) return e;
  // layer 1: dW1 from (da0, normalised state); dq += dX / std
  if ((e = cudaStreamWaitEvent(w, g.ev[7], 0)) != cudaSuccess) return e;
  if ((e = backward_first(net, q, g.da[0], L, B, ny, nx, g, part[1], dq, dparams, scale, w, s, ro)) != cudaSuccess)
    return e;
  if ((e = stream_after(g, 5, w, s)) != cudaSuccess) return e;
  return stream_after(g, 5, g.red, s);
}

cudaError_t backward_faces(const Net& net, const float* q, int B, int ny, int nx, const Acts& acts,
                           const float* sides, const float* ds, float* dq, float* dparams, float scale,
                           Grads& g, cudaStream_t s) {
  if (net.kind != NET_FACE || !acts.z[0]) return cudaErrorInvalidValue;
  const ParamLayout L = param_layout(NET_FACE);
  const long long plane = (long long)nx * ny, cells = (long long)B * plane;
  cudaError_t e;
  sides_to_raw_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(ds, sides, g.dr, plane, cells,
                                                                      net.std_[1], net.std_[2]);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cudaStream_t w = g.aux;   // dW beside dX, as in backward()
  ConvArgs a{};
  a.nx = nx;
  a.ny = ny;
  a.plane = plane;
  a.err = net.err;
  // (the reductions of an earlier call were joined into s: its buffers are
  // free, which the two buffer events restate from s, so that every wait
  // below refers to work of this call, as a graph capture requires)
  if ((e = cudaEventRecord(g.ev[6], s)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(g.ev[7], s)) != cudaSuccess) return e;
  if ((e = stream_after(g, 0, s, w)) != cudaSuccess) return e;
  // the reductions run on g.red; layers alternate between two partial
  // buffers, and a layer's partial sums wait for the reduction that last
  // read its buffer
  const RedOn ro{g.red, g.ev[8]};
  float* part[2] = {g.part, g.part2};
  // layer 4: dW4, db4 from (dr, a3); dX -> da[0] times GeLU'(z3)
  if ((e = cudaStreamWaitEvent(w, g.ev[6], 0)) != cudaSuccess) return e;
  if ((e = weight_grad<HID, N_OUT_FACE, 2>(acts.a[2], nullptr, g.dr, dparams + L.w[3], dparams + L.b[3],
                                           part[0], B, ny, nx, net, scale, w, ro)) != cudaSuccess)
    return e;
  if ((e = cudaEventRecord(g.ev[6], g.red)) != cudaSuccess) return e;
  a.x = g.dr;
  a.wpk = net.wb[3];
  a.z = acts.z[2];
  a.y = g.da[0];
  if ((e = launch_conv<2, HID, IN_ACT, OUT_GELU_GRAD>(a, B, s)) != cudaSuccess) return e;
  if ((e = stream_after(g, 1, s, w)) != cudaSuccess) return e;
  // layer 3: dW3 from (da0, a2); dX -> da[1] times GeLU'(z2)
  if ((e = cudaStreamWaitEvent(w, g.ev[7], 0)) != cudaSuccess) return e;
  if ((e = weight_grad<HID, HID, 4>(acts.a[1], nullptr, g.da[0], dparams + L.w[2], dparams + L.b[2],
                                    part[1], B, ny, nx, net, scale, w, ro)) != cudaSuccess)
    return e;
  if ((e = cudaEventRecord(g.ev[7], g.red)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(g.ev[2], w)) != cudaSuccess) return e;   // dW3 has read da[0]
  a.x = g.da[0];
  a.wpk = net.wb[2];
  a.z = acts.z[1];
  a.y = g.da[1];
  if ((e = launch_conv<CG_HID, HID, IN_ACT, OUT_GELU_GRAD>(a, B, s)) != cudaSuccess) return e;
  if ((e = stream_after(g, 3, s, w)) != cudaSuccess) return e;
  // layer 2: dW2 from (da1, a1); dX -> da[0] times GeLU'(z1)
  if ((e = cudaStreamWaitEvent(w, g.ev[6], 0)) != cudaSuccess) return e;
  if ((e = weight_grad<HID, HID, 4>(acts.a[0], nullptr, g.da[1], dparams + L.w[1], dparams + L.b[1],
                                    part[0], B, ny, nx, net, scale, w, ro)) != cudaSuccess)
    return e;
  if ((e = cudaEventRecord(g.ev[6], g.red)) != cudaSuccess) return e;
  a.x = g.da[1];
  a.wpk = net.wb[1];
  a.z = acts.z[0];
  a.y = g.da[0];
  if ((e = cudaStreamWaitEvent(s, g.ev[2], 0)) != cudaSuccess) return e;
  if ((e = launch_conv<CG_HID, HID, IN_ACT, OUT_GELU_GRAD>(a, B, s)) != cudaSuccess) return e;
  if ((e = stream_after(g, 4, s, w)) != cudaSuccess) return e;
  // layer 1: dW1 from (da0, normalised state); dq += dX / std
  if ((e = cudaStreamWaitEvent(w, g.ev[7], 0)) != cudaSuccess) return e;
  if ((e = backward_first(net, q, g.da[0], L, B, ny, nx, g, part[1], dq, dparams, scale, w, s, ro)) != cudaSuccess)
    return e;
  if ((e = stream_after(g, 5, w, s)) != cudaSuccess) return e;
  return stream_after(g, 5, g.red, s);
}

}  // namespace snk

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {

int net_alloc(fv_net* n, int kind) {
  snk::Net& N = n->n;
  N.kind = kind;
  const bool face = kind == snk::NET_FACE;
  cudaError_t e;
  if ((e = cudaMalloc(&N.params, sizeof(float) * snk::n_params(kind))) != cudaSuccess)
    return fvh::cuda_fail(e, "cudaMalloc(params)");
  const int fsz[4] = {9 * snk::CG_IN0 * snk::HID * 8, 9 * snk::CG_HID * snk::HID * 8,
                      9 * snk::CG_HID * snk::HID * 8,
                      9 * snk::CG_HID * (face ? snk::N_OUT_FACE_PAD : snk::N_OUT_PAD) * 8};
  for (int l = 0; l < 4; ++l)
    if ((e = cudaMalloc(&N.wf[l], 2 * fsz[l])) != cudaSuccess) return fvh::cuda_fail(e, "cudaMalloc(wf)");
  for (int l = 0; l < 4; ++l) {
    const int cg = snk::backward_groups(snk::param_layout(kind).cout[l]);
    const int nb = l == 0 ? snk::DQ_N : snk::HID;
    if ((e = cudaMalloc(&N.wb[l], 2 * 9 * cg * nb * 8)) != cudaSuccess)
      return fvh::cuda_fail(e, "cudaMalloc(wb)");
  }
  if (face) {
    // the row-pipelined operand layouts serve the fused stencil kernel only
  } else {
    if ((e = cudaMalloc(&N.w1g, 2 * snk::W1G_ELEMS)) != cudaSuccess) return fvh::cuda_fail(e, "cudaMalloc(w1g)");
    for (int l = 1; l < 3; ++l)
      if ((e = cudaMalloc(&N.wpair[l], 2 * fsz[l])) != cudaSuccess) return fvh::cuda_fail(e, "cudaMalloc(wpair)");
    if ((e = cudaMalloc(&N.w4ring, 2 * snk::W4R_ELEMS)) != cudaSuccess)
      return fvh::cuda_fail(e, "cudaMalloc(w4ring)");
  }
  if ((e = cudaMalloc(&N.err, sizeof(unsigned))) != cudaSuccess) return fvh::cuda_fail(e, "cudaMalloc(err)");
  if ((e = cudaMemset(N.err, 0, sizeof(unsigned))) != cudaSuccess) return fvh::cuda_fail(e, "cudaMemset");
  if ((e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return fvh::cuda_fail(e, "cudaStreamCreate");
  return FV_OK;
}

void net_free(fv_net* n) {
  if (!n) return;
  if (n->stream) cudaStreamSynchronize(n->stream);
  cudaFree(n->n.params);
  for (int l = 0; l < 4; ++l) {
    cudaFree(n->n.wf[l]);
    cudaFree(n->n.wb[l]);
  }
  cudaFree(n->n.w1g);
  for (int l = 1; l < 3; ++l) cudaFree(n->n.wpair[l]);
  cudaFree(n->n.w4ring);
  cudaFree(n->n.err);
  cudaFree(n->adam_m);
  cudaFree(n->adam_v);
  snk::acts_free(n->ws);
  snk::backward_free(n->bw);
  cudaFree(n->scratch);
  if (n->stream) cudaStreamDestroy(n->stream);
  delete n;
}

// Scratch of at least `floats` floats for the recomputed forward outputs.
cudaError_t scratch_reserve(fv_net* n, long long floats) {
  if (n->scratch_floats >= floats) return cudaSuccess;
  cudaFree(n->scratch);
  n->scratch = nullptr;
  n->scratch_floats = 0;
  cudaError_t e = cudaMalloc(&n->scratch, sizeof(float) * floats);
  if (e == cudaSuccess) n->scratch_floats = floats;
  return e;
}

int net_check_err(const fv_net* n) {
  unsigned h = 0;
  cudaError_t e = cudaMemcpy(&h, n->n.err, sizeof h, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fvh::cuda_fail(e, "reading the network error word");
  if (h) return fvh::fail(FV_ETIMEOUT, "a tensor-core wait gave up (bounded mbarrier wait)");
  return FV_OK;
}

}  // namespace

namespace fvs {
int net_check(const fv_net* n) { return net_check_err(n); }
}  // namespace fvs

namespace {

int create_net(int kind, const float* params, const float* norm, fv_net** out) {
  if (!out) return fvh::fail(FV_EINVAL, "null output");
  *out = nullptr;
  fv_net* n = new fv_net();
  int rc = net_alloc(n, kind);
  if (rc != FV_OK) {
    net_free(n);
    return rc;
  }
  if (norm) {
    for (int c = 0; c < 3; ++c) {
      n->n.mean[c] = norm[c];
      n->n.std_[c] = norm[3 + c];
      if (!(norm[3 + c] > 0.f)) {
        net_free(n);
        return fvh::fail(FV_EINVAL, "normalisation std must be > 0");
      }
    }
  }
  cudaError_t e;
  const size_t pbytes = sizeof(float) * snk::n_params(kind);
  if (params) {
    e = cudaMemcpy(n->n.params, params, pbytes, cudaMemcpyHostToDevice);
  } else {
    e = cudaMemset(n->n.params, 0, pbytes);
  }
  if (e == cudaSuccess) e = snk::repack(n->n, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) {
    net_free(n);
    return fvh::cuda_fail(e, "network creation");
  }
  *out = n;
  return FV_OK;
}

}  // namespace

extern "C" int stencil_net_create(const float* params, const float* norm, fv_net** out) {
  return create_net(snk::NET_STENCIL, params, norm, out);
}

extern "C" int face_net_create(const float* params, const float* norm, fv_net** out) {
  return create_net(snk::NET_FACE, params, norm, out);
}

extern "C" int fv_net_kind(const fv_net* n) { return n ? n->n.kind : -1; }

extern "C" int fv_net_num_params(const fv_net* n) { return n ? snk::n_params(n->n.kind) : 0; }

extern "C" int stencil_net_destroy(fv_net* n) {
  net_free(n);
  return FV_OK;
}

extern "C" int stencil_net_set_params(fv_net* n, const float* params, int loc) {
  if (!n || !params) return fvh::fail(FV_EINVAL, "null argument");
  FV_CUDA_TRY(cudaMemcpyAsync(n->n.params, params, sizeof(float) * snk::n_params(n->n.kind),
                              loc == FV_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              n->stream));
  FV_CUDA_TRY(snk::repack(n->n, n->stream));
  FV_CUDA_TRY(cudaStreamSynchronize(n->stream));
  return FV_OK;
}

extern "C" int stencil_net_get_params(const fv_net* n, float* params, int loc) {
  if (!n || !params) return fvh::fail(FV_EINVAL, "null argument");
  FV_CUDA_TRY(cudaStreamSynchronize(n->stream));
  FV_CUDA_TRY(cudaMemcpy(params, n->n.params, sizeof(float) * snk::n_params(n->n.kind),
                         loc == FV_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  return FV_OK;
}

extern "C" int stencil_net_forward(const fv_net* cn, const float* q, int B, int ny, int nx,
                                   float* coeffs, int raw, void* stream) {
  fv_net* n = const_cast<fv_net*>(cn);
  if (!n || !q || !coeffs) return fvh::fail(FV_EINVAL, "null argument");
  if (n->n.kind != snk::NET_STENCIL) return fvh::fail(FV_EINVAL, "not a stencil network (use face_net_forward)");
  if (B < 1 || ny < 1 || !snk::grid_supported(nx) || ((long long)nx * ny) % snk::TILE != 0)
    return fvh::fail(FV_EINVAL, "unsupported grid: nx must be 8, 16, 32, 64 or a multiple of 128, "
                                "and nx*ny a multiple of 128");
  cudaStream_t s = stream ? (cudaStream_t)stream : n->stream;
  FV_CUDA_TRY(snk::acts_reserve(n->ws, (long long)B * nx * ny));
  FV_CUDA_TRY(snk::forward(n->n, q, B, ny, nx, n->ws, raw ? nullptr : coeffs, raw ? coeffs : nullptr, s));
  FV_CUDA_TRY(cudaStreamSynchronize(s));
  return net_check_err(n);
}

extern "C" int face_net_forward(const fv_net* cn, const float* q, int B, int ny, int nx, float* sides,
                                int raw, void* stream) {
  fv_net* n = const_cast<fv_net*>(cn);
  if (!n || !q || !sides) return fvh::fail(FV_EINVAL, "null argument");
  if (n->n.kind != snk::NET_FACE) return fvh::fail(FV_EINVAL, "not a face-state network");
  if (B < 1 || ny < 1 || !snk::grid_supported(nx) || ((long long)nx * ny) % snk::TILE != 0)
    return fvh::fail(FV_EINVAL, "unsupported grid: nx must be 8, 16, 32, 64 or a multiple of 128, "
                                "and nx*ny a multiple of 128");
  cudaStream_t s = stream ? (cudaStream_t)stream : n->stream;
  FV_CUDA_TRY(snk::acts_reserve(n->ws, (long long)B * nx * ny));
  FV_CUDA_TRY(snk::forward_faces(n->n, q, B, ny, nx, n->ws, raw ? nullptr : sides, raw ? sides : nullptr, s));
  FV_CUDA_TRY(cudaStreamSynchronize(s));
  return net_check_err(n);
}

// Vector-Jacobian products of the two forwards: the forward is recomputed at
// q (activations into the network's workspace), then the hand-written
// backward of snk::backward / snk::backward_faces runs.
namespace {

int net_backward(fv_net* n, int kind, const float* q, int B, int ny, int nx, const float* dout, float* dq,
                 float* dparams, void* stream) {
  if (!n || !q || !dout || !dparams) return fvh::fail(FV_EINVAL, "null argument");
  if (n->n.kind != kind) return fvh::fail(FV_EINVAL, "network kind does not match the call");
  if (B < 1 || ny < 1 || !snk::grid_supported(nx) || ((long long)nx * ny) % snk::TILE != 0)
    return fvh::fail(FV_EINVAL, "unsupported grid: nx must be 8, 16, 32, 64 or a multiple of 128, "
                                "and nx*ny a multiple of 128");
  cudaStream_t s = stream ? (cudaStream_t)stream : n->stream;
  const long long cells = (long long)B * nx * ny;
  const bool face = kind == snk::NET_FACE;
  FV_CUDA_TRY(snk::acts_reserve(n->ws, cells, face));
  FV_CUDA_TRY(snk::backward_reserve(n->bw, cells, snk::backward_partials_floats(B, ny, nx)));
  FV_CUDA_TRY(scratch_reserve(n, cells * (face ? snk::N_OUT_FACE : snk::N_OUT)));
  if (face) {
    FV_CUDA_TRY(snk::forward_faces(n->n, q, B, ny, nx, n->ws, n->scratch, nullptr, s));
    FV_CUDA_TRY(snk::backward_faces(n->n, q, B, ny, nx, n->ws, n->scratch, dout, dq, dparams, 1.f, n->bw, s));
  } else {
    FV_CUDA_TRY(snk::forward(n->n, q, B, ny, nx, n->ws, n->scratch, nullptr, s));
    FV_CUDA_TRY(snk::backward(n->n, q, B, ny, nx, n->ws, dout, dq, dparams, 1.f, n->bw, s));
  }
  FV_CUDA_TRY(cudaStreamSynchronize(s));
  return net_check_err(n);
}

}  // namespace

extern "C" int stencil_net_backward(fv_net* n, const float* q, int B, int ny, int nx, const float* dcoeffs,
                                    float* dq, float* dparams, void* stream) {
  return net_backward(n, snk::NET_STENCIL, q, B, ny, nx, dcoeffs, dq, dparams, stream);
}

extern "C" int face_net_backward(fv_net* n, const float* q, int B, int ny, int nx, const float* dsides,
                                 float* dq, float* dparams, void* stream) {
  return net_backward(n, snk::NET_FACE, q, B, ny, nx, dsides, dq, dparams, stream);
}
