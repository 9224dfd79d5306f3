// fv_fused.cu — the learned-stencil SSP-RK2 stage as one persistent kernel.
//
// One launch = one Runge-Kutta stage (Eq. 2.19) of the learned step (Section
// 2.5.3, fourth approach) over every member: CNN (four 3x3 periodic
// convolutions on tcgen05, BF16 operands, FP32 accumulators in TMEM), the
// sum-to-one normalisation of the 36 outputs, the learned face states with
// their minmod fallback, the HLL fluxes (Eq. 2.15, rotated on y faces, Eq.
// 2.24), the flux divergence (Eq. 2.23), the RK combine and, in stage 2, the
// Courant-rate reduction for the next dt (Eq. 2.10).  Activations and
// coefficients never leave the SM: HBM sees the stage input, q^n in stage 2
// and the stage output, as in the plain step.
//
// Work decomposition.  A cluster of CS = nx / 128 CTAs (one per SM) owns whole
// grid rows: CTA r of the cluster owns columns [128 r, 128 r + 128).  The
// rows of all members, concatenated, are split into 2 x (number of clusters)
// contiguous ranges, two per cluster ("streams").  A stream marches down its
// rows; a tick processes one row at every layer of the pipeline:
//   MMA(tick):  layer 1 output row t-1, and for layers 2, 3, 4 the completion
//               of one output row and the start of the next (below);
//   EPI(tick):  drain the finished accumulators (bias, ReLU, BF16) into the
//               next layer's input rows; layer 4 gives the coefficients of row
//               t-7 and, straight from registers, that row's x-face fluxes and
//               its north y-face fluxes; update row t-8; build the layer-1
//               input of row t+1 and stage the FP32 state row t-4.
// The two streams alternate: in each phase the tensor core works on one
// stream's tick while the CUDA cores drain the other's.
//
// Threads: warpgroups 0 and 1 drain TMEM (each thread one TMEM lane = one
// column) and compute the faces, and warpgroup 0 updates the finished row
// while it waits for the MMAs; warpgroup 2's first warp issues the MMAs (one
// lane), its other three warps stage the state rows and the layer-1 input and
// place the halo columns received from the neighbours.  They hand work to
// each other through mbarriers (see `phase`), not through block or cluster
// barriers.
//
// Layers 2-4 keep two input rows and two adjacent accumulators each: slot 0
// holds the row started at the previous tick (taps ky = 0 and 1 summed), slot
// 1 the row started now.  When input row k arrives, six MMAs of the taps
// ky = 0 on row k-1 start slot 1, and six MMAs with the taps ky = 2 and ky = 1
// stacked along N (one read of row k, N = 64 or 96) complete slot 0 and add
// to slot 1; after the drain, slot 1 moves to slot 0.  An output row thus sums
// its taps in the order ky = 0, 1, 2 (kx and channel groups inner), the same
// order as the two-pass CNN.  Layer 1 reads the three x taps of the state
// gathered into one K = 16 operand (9 used channels) and sums three dy taps.
// The 1-cell x halo of every hidden layer comes from the neighbouring CTA of
// the cluster (asynchronous distributed-shared-memory copies; the periodic
// wrap for CS = 1), and so does the flux through the west face of column 0.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fv_common.cuh"
#include "fv_internal.h"
#include "fv_learned.cuh"
#include "stencil_net.cuh"
#include "tc_common.cuh"

namespace fvk {
namespace fused {

constexpr int EPI_THREADS = 256;        // 2 warpgroups that drain TMEM
constexpr int NT = EPI_THREADS + 128;   // + the update / staging warpgroup
constexpr int ISSUE_WARP = EPI_THREADS / 32;
constexpr int W = 128;                  // columns per CTA = MMA M
constexpr int FP = W + 2;               // hidden-layer input frame (1-cell halo)
constexpr int QF = W + 4;               // FP32 state frame (2-cell halo)
constexpr int MAX_CS = 8;               // portable cluster size
constexpr int TICKS_AHEAD = 11;         // ticks before the first updated row
constexpr uint32_t WAIT_ITERS = 1u << 22;

// shared memory (bytes)
constexpr int L1_SLOT = 2 * W * 16;                 // [2 groups][128][8 BF16]
constexpr int HID_SLOT = 4 * FP * 16;               // [4 groups][130][8 BF16]
constexpr int Q_SLOT = 3 * QF * 4;                  // [3 vars][132] FP32
constexpr int F_SLOT = 1552;                        // [3 vars][129] FP32, padded
constexpr int G_SLOT = 3 * W * 4;                   // [3 vars][128] FP32
constexpr int QN_SLOT = 3 * W * 4;                  // [3 vars][128] FP32: q^n of the next update
constexpr int OFF_L1 = 0;                           // 3 slots
constexpr int OFF_IN = OFF_L1 + 3 * L1_SLOT;        // layers 2..4 inputs, 2 slots each
constexpr int OFF_Q = OFF_IN + 3 * 2 * HID_SLOT;    // 5 slots
constexpr int OFF_F = OFF_Q + 5 * Q_SLOT;           // 2 slots
constexpr int OFF_G = OFF_F + 2 * F_SLOT;           // 3 slots
constexpr int OFF_QN = OFF_G + 3 * G_SLOT;          // 1 slot
constexpr int OFF_FXO = OFF_QN + QN_SLOT;           // [2][4] FP32: east-face flux of column 127, sent east
constexpr int OFF_FXI = OFF_FXO + 32;               // [2][4] FP32: west-face flux of column 0, received
// halo columns of the three hidden-layer input rows, [side][layer][group] x
// 16 bytes: sent (side 0 = column 0, for the west neighbour; 1 = column
// W - 1, for the east neighbour) and received (side 0 = from the west
// neighbour, for position 0; 1 = from the east neighbour, for position W + 1)
constexpr int HALO_SIDE = 3 * 4 * 16;
constexpr int OFF_HOUT = OFF_FXI + 32;
constexpr int OFF_HIN = OFF_HOUT + 2 * HALO_SIDE;
// FP32 state row t+1 of the next tick's layer-1 input, [3 vars][W + 8], frame
// position p = column - X0 + 4 (16-byte aligned interior)
constexpr int RAWF = W + 8;
constexpr int OFF_RAW = OFF_HIN + 2 * HALO_SIDE;
constexpr int STREAM_BYTES = OFF_RAW + 3 * RAWF * 4;

constexpr int W1_BYTES = snk::W1G_ELEMS * 2;                       // 3072
constexpr int WH_BYTES = 9 * snk::CG_HID * snk::HID * 16;          // 18432
constexpr int W4_BYTES = snk::W4R_ELEMS * 2;                       // 24576
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + W1_BYTES;
constexpr int OFF_W3 = OFF_W2 + WH_BYTES;
constexpr int OFF_W4 = OFF_W3 + WH_BYTES;
constexpr int OFF_STREAMS = OFF_W4 + W4_BYTES;
// biases of layers 1..3, then of layer 4's 24 differences (b[3 s + j] - b[3 s + 2])
constexpr int N_BIAS = 3 * snk::HID + snk::W4R_BLOCK;
constexpr int OFF_BIAS = OFF_STREAMS + 2 * STREAM_BYTES;
// mbarriers: [0..1] MMAs of stream s done, [2..3] inputs of the next tick of
// stream s ready, [4..7] tick n of stream s done (index 4 + 2 s + (n & 1)),
// [8..9] the neighbours' halo columns of stream s received
constexpr int OFF_MBAR = OFF_BIAS + ((N_BIAS * 4 + 15) / 16) * 16;
constexpr int OFF_TSLOT = OFF_MBAR + 10 * 8;
constexpr int OFF_RED = OFF_TSLOT + 16;
constexpr int SMEM_BYTES = OFF_RED + 32 * 4;

static_assert(STREAM_BYTES % 16 == 0 && OFF_STREAMS % 16 == 0, "16-byte aligned operands");
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");

// TMEM columns of one stream (two streams: 2 x 256 = 512)
constexpr uint32_t TCOLS = 512;
constexpr uint32_t ACC1 = 0;
// layer 0..1 = layers 2..3; slot 0 and slot 1 are adjacent
__host__ __device__ constexpr uint32_t acc_col(int layer, int slot) { return 32u + 64u * layer + 32u * slot; }
// Layer 4: a ring of three 24-column slots (the 24 stencil differences of
// one output row each), then 8 columns that the 80-wide MMAs also write and
// nothing reads.  The row completed at tick n of a stream is in slot n % 3.
constexpr uint32_t ACC4 = 160;
constexpr uint32_t R4 = snk::W4R_BLOCK;                // 24
constexpr uint32_t N4 = 3 * R4 + 8;                    // 80 (N multiple of 16)

struct Args {
  const float* qin;
  const float* qn;
  float* qout;
  const uint16_t* w1g;
  const uint16_t* w2;
  const uint16_t* w3;
  const uint16_t* w4;
  const float* params;
  int bias_off[4];
  float mean[3], rstd[3];
  const float* hmin;
  Ctrl* ctrl;
  const DtParams* dp;
  int nx, ny, cs;
  long long plane, member;
  long long rows;          // B * ny
  long long nstreams;      // 2 x clusters
  float rdx, rdy, g;
  unsigned* err;
  int hy;                  // ring rows of a subdomain: outside the CFL reduction
};

// ---------------------------------------------------------------------------
// Cluster, TMEM and copy helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t map_cta(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
// Arrive on a local mbarrier (release at CTA scope), optionally raising the
// number of bytes its current phase still waits for.
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(mbar)),
               "r"(bytes)
               : "memory");
}
// Asynchronous copy of `bytes` (a multiple of 16) from this CTA's shared
// memory at `src` to the same offset as `dst` in CTA `rank` of the cluster; completes (bytes) on that
// CTA's mbarrier at the offset of `mbar`.  The source must have been made
// visible to the async proxy (fence.proxy.async) by this thread.
__device__ __forceinline__ void copy_to_cta(const void* dst, const void* src, uint32_t bytes, uint64_t* mbar,
                                            uint32_t rank) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   map_cta(tc::smem_u32(dst), rank)),
               "r"(tc::smem_u32(src)), "r"(bytes), "r"(map_cta(tc::smem_u32(mbar), rank))
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(tc::smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// Arrive on the mbarrier at the same shared-memory offset in every CTA of
// `mask` once this thread's earlier tcgen05.mma have completed.
__device__ __forceinline__ void commit_multicast(uint64_t* mbar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n"
      ::"r"(tc::smem_u32(mbar)), "h"(mask)
      : "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n"
               ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                 "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])),
                 "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const float (&v)[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3]))
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16};\n"
      ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::smem_u32(smem)), "l"(gmem)
               : "memory");
}
// Periodic index for rows (any offset: 32-bit remainder) and for columns
// (offsets of at most one period: two compares).
__device__ __forceinline__ int wrap_row(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}
__device__ __forceinline__ int wrap_col(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Index of the stream whose row range holds global row r (ranges are
// [k R / S, (k + 1) R / S)).
__device__ __forceinline__ long long stream_of_row(long long r, long long R, long long S) {
  return ((r + 1) * S - 1) / R;
}

// Per-thread copy of a stream's position; every thread updates it the same way.
struct Stream {
  long long g, g_end;      // next row of the range (concatenated rows), end of range
  int b, u0, u1;           // current segment: member and its rows [u0, u1)
  int tau, ntau;           // tick within the segment
  bool active, pending;    // has a segment; MMAs issued and not yet drained
  uint32_t parity;         // next phase of the stream's MMA mbarrier
  uint32_t nt;             // ticks drained so far (all segments)
  float dt, hmin;
  float amax;
  unsigned bad;
};

// q^n of cell m of the row the next tick of this stream updates (stage 2),
// copied into the stream's q^n slot one tick ahead of its use (cp.async: no
// registers held across the phases).
__device__ __forceinline__ void fetch_qn(float* qnb, const Args& a, int b, int u, int X0, int m) {
  const long long off = (long long)b * a.member + (long long)u * a.nx + X0 + m;
#pragma unroll
  for (int c = 0; c < 3; ++c) cp_async4(qnb + c * W + m, a.qn + off + c * a.plane);
}

// Layer-1 input at position m: the normalised state of the cells m-1, m,
// m+1 as channel 3 kx + var (x = (q - mean) / scale, as in the two-pass CNN),
// BF16, 9 of 16 channels used.
__device__ __forceinline__ void prep_l1_pos(uint8_t* slot, const Args& a, const float (&q)[9], int m) {
  float ch[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) ch[c] = (q[c] - a.mean[c % 3]) * a.rstd[c % 3];
  const uint4 g0 = make_uint4(pack_bf16x2(ch[0], ch[1]), pack_bf16x2(ch[2], ch[3]),
                              pack_bf16x2(ch[4], ch[5]), pack_bf16x2(ch[6], ch[7]));
  const uint4 g1 = make_uint4(pack_bf16x2(ch[8], 0.f), 0u, 0u, 0u);
  *reinterpret_cast<uint4*>(slot + m * 16) = g0;
  *reinterpret_cast<uint4*>(slot + (W + m) * 16) = g1;
}

// The layer-1 input row `row`, positions k and k + n (n >= 64): the loads of
// both positions first, then the stores.
__device__ __forceinline__ void load_l1_row(float (&q)[2][9], const Args& a, const float* qb, int row,
                                            int X0, int k, int n) {
  const float* base = qb + (long long)wrap_row(row, a.ny) * a.nx;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int m = k + r * n;
    if (m < W) {
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int col = wrap_col(X0 + m + kx - 1, a.nx);
#pragma unroll
        for (int v = 0; v < 3; ++v) q[r][3 * kx + v] = base[v * a.plane + col];
      }
    }
  }
}
__device__ __forceinline__ void store_l1_row(uint8_t* slot, const Args& a, const float (&q)[2][9], int k,
                                             int n) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int m = k + r * n;
    if (m < W) prep_l1_pos(slot, a, q[r], m);
  }
}

// The raw state row `row` (three variables, columns X0 - 1 .. X0 + W) into
// the stream's raw row, by the 96 staging threads (k = 0..95): one 16-byte
// copy of the interior each, and the two halo cells of each variable.
__device__ __forceinline__ void fetch_raw_row(float* raw, const Args& a, const float* qb, int row, int X0,
                                              int k) {
  const float* base = qb + (long long)wrap_row(row, a.ny) * a.nx;
  const int v = k >> 5, j = k & 31;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::smem_u32(raw + v * RAWF + 4 + 4 * j)),
               "l"(base + v * a.plane + X0 + 4 * j)
               : "memory");
  if (k < 6) {
    const int hv = k >> 1, east = k & 1;
    cp_async4(raw + hv * RAWF + (east ? 4 + W : 3), base + hv * a.plane + wrap_col(east ? X0 + W : X0 - 1, a.nx));
  }
}

// The layer-1 input row from the raw row, positions k and k + n (n >= 64).
__device__ __forceinline__ void build_l1_row(uint8_t* slot, const float* raw, const Args& a, int k, int n) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int m = k + r * n;
    if (m < W) {
      float q[9];
#pragma unroll
      for (int kx = 0; kx < 3; ++kx)
#pragma unroll
        for (int v = 0; v < 3; ++v) q[3 * kx + v] = raw[v * RAWF + m + 3 + kx];
      prep_l1_pos(slot, a, q, m);
    }
  }
}

// FP32 state row with a 2-cell periodic halo: frame position p is column
// X0 - 2 + p; elements k, k + n, ... (n >= 96: at most five per thread),
// copied with cp.async (the caller commits and waits).
__device__ __forceinline__ void load_q_row(float* slot, const Args& a, const float* qb, int row,
                                           int X0, int k, int n) {
  const float* base = qb + (long long)wrap_row(row, a.ny) * a.nx;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int idx = k + i * n;
    if (idx < 3 * QF) {
      const int c = idx / QF, p = idx - c * QF;
      cp_async4(slot + idx, base + c * a.plane + wrap_col(X0 - 2 + p, a.nx));
    }
  }
}

// Bring a state row (three variables, this CTA's columns) into L2 ahead of use.
__device__ __forceinline__ void prefetch_row(const Args& a, const float* qb, int row, int X0, int k) {
  if (k < 3 * 4) {
    const int v = k / 4, seg = k % 4;    // 4 x 128-byte lines per variable and row
    const float* p = qb + v * a.plane + (long long)wrap_row(row, a.ny) * a.nx + X0 + 32 * seg;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  }
}

// Bias, ReLU and BF16 of 16 accumulator columns (channel groups 2 wg, 2 wg + 1)
// into position m + 1 of the next layer's input row; the edge columns also
// into the layer's part of the halo-out buffer.
__device__ __forceinline__ void drain_hidden(uint32_t taddr, const float* bias, uint8_t* dst, uint8_t* hout,
                                             int m, int wg) {
  float v[16];
  tc::tmem_ld16(taddr + 16 * wg, v);
#pragma unroll
  for (int gg = 0; gg < 2; ++gg) {
    const int g = 2 * wg + gg;
    uint32_t pk[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 8 * gg + 2 * j;
      pk[j] = pack_bf16x2(fmaxf(v[c] + bias[8 * g + 2 * j], 0.f),
                          fmaxf(v[c + 1] + bias[8 * g + 2 * j + 1], 0.f));
    }
    const uint4 val = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4*>(dst + g * FP * 16 + (m + 1) * 16) = val;
    if (m == 0 || m == W - 1) *reinterpret_cast<uint4*>(hout + (m ? HALO_SIDE : 0) + g * 16) = val;
  }
}

// The 18 normalised coefficients of one direction (dir 0: stencils 0..5 =
// x, dir 1: 6..11 = y) of this lane's cell from the layer-4 ring slot `taddr`:
// per 3-tap stencil the raw outputs r enter only through r - mean(r), which
// the differences s1 = r0 - r2, s2 = r1 - r2 (+ their biases) determine:
//   r0 - m = (2 s1 - s2) / 3,  r1 - m = (2 s2 - s1) / 3,  r2 - m = -(s1 + s2) / 3,
// and w = e_centre + r - mean(r) as in the two-pass CNN's epilogue.
__device__ __forceinline__ void drain_coeffs(uint32_t taddr, const float* bias, int dir, float (&wd)[18]) {
  // columns 8 dir .. 8 dir + 15 (differences 12 dir .. 12 dir + 11 used)
  float v[16];
  tc::tmem_ld16(taddr + 8 * dir, v);
  const float third = 1.f / 3.f;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const float x1 = dir ? v[4 + 2 * s] : v[2 * s];
    const float x2 = dir ? v[5 + 2 * s] : v[2 * s + 1];
    const float s1 = x1 + bias[12 * dir + 2 * s];
    const float s2 = x2 + bias[12 * dir + 2 * s + 1];
    wd[3 * s] = (2.f * s1 - s2) * third;
    wd[3 * s + 1] = 1.f + (2.f * s2 - s1) * third;
    wd[3 * s + 2] = -(s1 + s2) * third;
  }
}

// Once every slot-0 read of the tick is done: the row started this tick
// (slot 1) becomes the row to complete next tick (slot 0), for layers 2 and
// 3 (warpgroup 0 moves columns 0-15, warpgroup 1 columns 16-31, each thread
// its own TMEM lane), and the layer-4 ring slot drained in this tick is
// cleared (warpgroup 0 its columns 0-11, warpgroup 1 12-23): the next tick's
// MMAs start a new row in it by accumulating.
__device__ __forceinline__ void move_slots(uint32_t tm, uint32_t ring_slot, int wg) {
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    float v[16];
    tc::tmem_ld16(tm + acc_col(l, 1) + 16 * wg, v);
    tmem_st16(tm + acc_col(l, 0) + 16 * wg, v);
  }
  const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, z4[4] = {0.f, 0.f, 0.f, 0.f};
  tmem_st8(ring_slot + 12 * wg, z8);
  tmem_st4(ring_slot + 12 * wg + 8, z4);
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// Move a stream to its next segment whose member still has work; false when
// the range is exhausted.  Every thread runs this with the same inputs.
__device__ bool next_segment(Stream& S, const Args& a, uint32_t crank) {
  while (S.g < S.g_end) {
    const int b = (int)(S.g / a.ny);
    const int u0 = (int)(S.g - (long long)b * a.ny);
    const long long left = S.g_end - S.g;
    const int u1 = (int)((long long)(a.ny - u0) < left ? a.ny : u0 + left);
    S.g = (long long)b * a.ny + u1;
    Ctrl* c = a.ctrl + b;
    if (*reinterpret_cast<volatile unsigned*>(&c->done)) {
      // a stage attempted after REPLAY ran out (flagged once per member)
      if (c->exhausted && u0 == 0 && crank == 0 && threadIdx.x == 0)
        atomicOr(&c->health, FV_HEALTH_REPLAY_END);
      continue;
    }
    S.b = b;
    S.u0 = u0;
    S.u1 = u1;
    S.tau = 0;
    S.ntau = u1 - u0 + TICKS_AHEAD;
    S.dt = (float)c->dt;
    S.hmin = a.hmin[b];
    S.amax = 0.f;
    S.bad = 0u;
    return true;
  }
  return false;
}

// Start of a segment: layer-1 inputs of rows u0-5, u0-4, u0-3 (slots 0, 1,
// 2), one row per warpgroup, and the raw row u0-2.  (The issuing warp takes no part: it has not
// waited for the MMAs that read these slots.)
// (`work` false: only the staging threads' named barrier.)
__device__ __forceinline__ void segment_prologue(const Stream& S, uint8_t* sbuf, const Args& a,
                                                 int X0, int m, int wg, bool work) {
  if (wg == 2 && m < 32) return;
  const int k = wg == 2 ? m - 32 : m, n = wg == 2 ? W - 32 : W;
  const float* qb = a.qin + (long long)S.b * a.member;
  if (work) {
    float q[2][9];
    load_l1_row(q, a, qb, S.u0 - 5 + wg, X0, k, n);
    store_l1_row(sbuf + OFF_L1 + wg * L1_SLOT, a, q, k, n);
  }
  if (wg == 2) {
    // the raw row of the first tick's layer-1 input, visible to all staging
    // threads before they leave
    if (work) {
      fetch_raw_row(reinterpret_cast<float*>(sbuf + OFF_RAW), a, qb, S.u0 - 2, X0, k);
      asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    asm volatile("bar.sync 5, 96;" ::: "memory");
  }
}

// Shared-memory descriptors of the operands; a slot or tap offset is added to
// the start-address field (bits 0-13, address / 16; shared addresses stay
// below 256 KB, so the field never overflows).
struct Descs {
  uint64_t a_l1, a_in, b_w1;
  uint64_t b_ky0[2], b_pair[2];   // layers 2..3: taps ky = 0, and ky = 2 | ky = 1 stacked
  uint64_t b_ring;                // layer 4: tap blocks ky = 2, 1, 0, 2, 1
};
__device__ __forceinline__ uint64_t dplus(uint64_t d, uint32_t bytes) { return d + (bytes >> 4); }

// tcgen05.mma with both shared-memory descriptors given by their low words:
// every operand of this kernel has the same high word (stride between
// 8-row core matrices 128 bytes, descriptor version 1), so only the start
// address and leading-dimension fields vary; `acc` is a compile-time flag.
template <bool ACC, uint32_t IDESC>
__device__ __forceinline__ void mma_lo(uint32_t d_tmem, uint32_t a_lo, uint32_t b_lo) {
  constexpr uint32_t hi = (128u >> 4) | (1u << 14);
  asm volatile(
      "{\n.reg .b64 da, db;\n.reg .pred p;\nmov.b64 da, {%1, %3};\nmov.b64 db, {%2, %3};\n"
      "setp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n}\n"
      ::"r"(d_tmem), "r"(a_lo), "r"(b_lo), "n"(hi), "n"(ACC ? 1 : 0), "n"(IDESC)
      : "memory");
}

// All MMAs of one tick of one stream (issued by one thread), then a commit
// to the stream's mbarrier in this CTA and its neighbours; `tm`: the
// stream's first TMEM column.
__device__ __forceinline__ void issue_tick(const Descs& D, uint32_t tm, int tau, uint32_t nt, uint64_t* mbar,
                                           uint16_t mask) {
  constexpr uint32_t id32 = tc::idesc_bf16_f32(W, snk::HID);
  constexpr uint32_t id64 = tc::idesc_bf16_f32(W, 2 * snk::HID);
  constexpr uint32_t id80 = tc::idesc_bf16_f32(W, N4);
  // layers 2..4: new input row in slot (tau+1)&1, previous one in slot tau&1
  const uint32_t s_new = (uint32_t)((tau + 1) & 1), s_prev = (uint32_t)(tau & 1);
  // low descriptor words (start address in 16-byte units in bits 0-13)
  const uint32_t in_lo = (uint32_t)D.a_in, l1_lo = (uint32_t)D.a_l1, w1_lo = (uint32_t)D.b_w1;
  uint32_t a_new[3], a_prev[2], b0[2], bp[2];
#pragma unroll
  for (int l = 0; l < 3; ++l) a_new[l] = in_lo + (((uint32_t)(l * 2 * HID_SLOT) + s_new * HID_SLOT) >> 4);
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    a_prev[l] = in_lo + (((uint32_t)(l * 2 * HID_SLOT) + s_prev * HID_SLOT) >> 4);
    b0[l] = (uint32_t)D.b_ky0[l];
    bp[l] = (uint32_t)D.b_pair[l];
  }
  // Layer 4's window covers ring slots 0, 1, 2; slot nt % 3 completes its row
  // (tap ky = 2), slot (nt + 1) % 3 adds ky = 1, slot (nt + 2) % 3 starts a
  // row (ky = 0): tap blocks 2,1,0 / 0,2,1 / 1,0,2 start at block 0 / 2 / 1.
  const uint32_t r3 = nt % 3u;
  const uint32_t ring_lo = (uint32_t)D.b_ring + (r3 == 0 ? 0u : (r3 == 1 ? 2u : 1u)) * R4;
  // Steps 0-5: layer 1 (taps ky on input rows t-2, t-1, t) and, for layers 2
  // and 3, the taps ky = 0 on the previous row into slot 1; steps 6-11: the
  // stacked taps ky = 2 | ky = 1 on the new row into slot 0 | slot 1, and
  // layer 4's three stacked taps on its new row into the ring.  Layers are
  // interleaved so that consecutive MMAs target different accumulators.
  // accumulator columns of this stream
  const uint32_t d1 = tm + ACC1, d4 = tm + ACC4;
  uint32_t dn[2], dc[2];
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    dn[l] = tm + acc_col(l, 1);
    dc[l] = tm + acc_col(l, 0);
  }
  const uint32_t s0 = (uint32_t)(tau % 3);
  const uint32_t l1s[3] = {s0, s0 == 2 ? 0u : s0 + 1, s0 == 0 ? 2u : s0 - 1};   // (tau + i) % 3
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    if (i < 3) {
      const uint32_t a = l1_lo + l1s[i] * (L1_SLOT >> 4), b = w1_lo + (uint32_t)(i * 2 * snk::HID);
      if (i == 0) mma_lo<false, id32>(d1, a, b);
      else mma_lo<true, id32>(d1, a, b);
    }
    const int j = i % 6, kx = j / 2, ks = j % 2;
    const uint32_t aoff = (uint32_t)(2 * ks * FP + kx);   // 16-byte units
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      constexpr uint32_t N = snk::HID;
      if (i < 6) {
        const uint32_t b = b0[l] + (uint32_t)((kx * 4 + 2 * ks) * N);
        if (i == 0) mma_lo<false, id32>(dn[l], a_prev[l] + aoff, b);
        else mma_lo<true, id32>(dn[l], a_prev[l] + aoff, b);
      } else {
        mma_lo<true, id64>(dc[l], a_new[l] + aoff, bp[l] + (uint32_t)((kx * 4 + 2 * ks) * 2 * N));
      }
    }
    if (i >= 6) mma_lo<true, id80>(d4, a_new[2] + aoff, ring_lo + (uint32_t)((kx * 4 + 2 * ks) * snk::W4R_ROWS));
  }
  // completion is signalled to this CTA and to its neighbours, which write
  // into the rows these MMAs read only after it
  commit_multicast(mbar, mask);
}

// Per-thread kernel context.
struct Ctx {
  uint8_t* smem;
  const float* bias;
  uint64_t* mbar;
  unsigned* red;
  uint32_t tmem;
  Descs D;                // operands of stream 0 (stream 1: + STREAM_BYTES)
  int tid, m, wg, X0;
  uint32_t lane_off, west, east, crank;
  uint16_t commit_mask;
  bool issuer, failed;
};

// Update of cell m of row u = t - 8 from the fluxes of the two previous
// ticks (nothing here depends on this tick's MMAs; run by draining
// warpgroup 0 while it waits for them), and the copy of q^n for the cell the
// next tick updates.
template <int STAGE>
__device__ __forceinline__ void update_cell(Stream& Q, uint8_t* sbuf, const Args& a, const Ctx& X, int m) {
  const int tau = Q.tau;
  const int t = Q.u0 - 3 + tau;
  const float* qring = reinterpret_cast<const float*>(sbuf + OFF_Q);
  const float* Fb = reinterpret_cast<const float*>(sbuf + OFF_F);
  const float* Gb = reinterpret_cast<const float*>(sbuf + OFF_G);
  float* qnb = reinterpret_cast<float*>(sbuf + OFF_QN);
  if (tau >= TICKS_AHEAD) {
    // this thread's copies of q^n (issued one tick of this stream back)
    if (STAGE == 2) asm volatile("cp.async.wait_all;\n" ::: "memory");
    const int u = t - 8;
    const float* Fo = Fb + ((tau + 1) & 1) * (F_SLOT / 4);
    const float* Fw = reinterpret_cast<const float*>(sbuf + OFF_FXI) + ((Q.nt + 1) & 1) * 4;
    const float* Gs = Gb + ((tau + 1) % 3) * (G_SLOT / 4);
    const float* Gn = Gb + ((tau + 2) % 3) * (G_SLOT / 4);
    const float* qu = qring + ((tau + 1) % 5) * (3 * QF);
    const long long off = (long long)Q.b * a.member + (long long)u * a.nx + X.X0 + m;
    float out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // the west face of column 0 is the west neighbour's east face
      const float fw = m == 0 ? Fw[c] : Fo[c * (W + 1) + m];
      const float Lc = divergence<float>(fw, Fo[c * (W + 1) + m + 1], Gs[c * W + m], Gn[c * W + m], a.rdx,
                                         a.rdy);
      const float q = qu[c * QF + m + 2];
      out[c] = STAGE == 1 ? rk_stage1<float>(q, Q.dt, Lc) : rk_stage2<float>(qnb[c * W + m], q, 0.5f * Q.dt, Lc);
      a.qout[off + c * a.plane] = out[c];
    }
    if (STAGE == 2 && u >= a.hy && u < a.ny - a.hy)
      Q.amax = fmaxf(Q.amax, cell_rate_swe(out[0], out[1], out[2], a.g, a.rdx, a.rdy, Q.bad));
  }
  if (STAGE == 2 && tau + 1 >= TICKS_AHEAD && tau + 1 < Q.ntau) {
    fetch_qn(qnb, a, Q.b, t - 7, X.X0, m);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
}

// The TMEM-draining warpgroups' part of tick Q.tau (after its MMAs), first
// half: the finished hidden accumulators into the next layer's input rows
// (slot tau & 1), which the next tick's MMAs and the halo copies read through
// the async proxy.  Then (in the caller) the layer-4 coefficients of row
// j = t - 7 and the slot move; after those the next tick may be issued.
__device__ __forceinline__ void drain_rows(const Stream& Q, uint8_t* sbuf, uint32_t tm, const Ctx& X) {
  const int m = X.m, wg = X.wg;
  const float* bias = X.bias;
  uint8_t* in = sbuf + OFF_IN + (Q.tau & 1) * HID_SLOT;
  uint8_t* hout = sbuf + OFF_HOUT;
  drain_hidden(tm + ACC1, bias, in, hout, m, wg);
  drain_hidden(tm + acc_col(0, 0), bias + snk::HID, in + 2 * HID_SLOT, hout + 64, m, wg);
  drain_hidden(tm + acc_col(1, 0), bias + 2 * snk::HID, in + 4 * HID_SLOT, hout + 128, m, wg);
  tc::fence_proxy_async_smem();
}

// The edge columns of the rows just drained go to the neighbours: two copies
// of 192 bytes (threads 0 and 1, after every draining warp wrote its rows)
// into their halo-in buffers, completing on their "halos received" mbarrier
// of the stream.
__device__ __forceinline__ void send_halos(uint8_t* sbuf, uint64_t* halo_in, const Ctx& X) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) copy_to_cta(sbuf + OFF_HIN + HALO_SIDE, sbuf + OFF_HOUT, HALO_SIDE, halo_in, X.west);
  if (lane == 1) copy_to_cta(sbuf + OFF_HIN, sbuf + OFF_HOUT + HALO_SIDE, HALO_SIDE, halo_in, X.east);
}

// Staging warp 10, every tick: once the neighbours' halo columns of tick
// Q.tau have landed, place them at positions 0 and W + 1 of the rows drained
// in this tick (slot tau & 1), where the next tick's MMAs read them.
__device__ __forceinline__ bool place_halos(const Stream& Q, uint8_t* sbuf, uint64_t* halo_in, bool ok) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) mbar_arrive_expect_tx(halo_in, 2 * HALO_SIDE);
  if (ok) ok = tc::mbar_wait_bounded(halo_in, Q.nt & 1, WAIT_ITERS);
  if (ok && lane < 24) {
    const int side = lane / 12, l = (lane >> 2) % 3, g = lane & 3;
    uint8_t* row = sbuf + OFF_IN + 2 * l * HID_SLOT + (Q.tau & 1) * HID_SLOT + g * FP * 16;
    *reinterpret_cast<uint4*>(row + (side ? FP - 1 : 0) * 16) =
        *reinterpret_cast<const uint4*>(sbuf + OFF_HIN + lane * 16);
  }
  tc::fence_proxy_async_smem();
  return ok;
}

// Second half: the faces row j owns from the coefficients `wd` and the
// staged state rows; x-face fluxes into F slot tau & 1 (the east face of
// column W - 1 also to the east neighbour), y-face fluxes into G slot tau % 3.
__device__ __forceinline__ void epilogue_faces(const Stream& Q, uint8_t* sbuf, const Args& a, const Ctx& X,
                                               uint64_t* tick_done, const float (&wd)[18]) {
  const int m = X.m, wg = X.wg;
  const int tau = Q.tau;
  float* qring = reinterpret_cast<float*>(sbuf + OFF_Q);
  float* Fb = reinterpret_cast<float*>(sbuf + OFF_F);
  float* Gb = reinterpret_cast<float*>(sbuf + OFF_G);
  const float* qj = qring + ((tau + 2) % 5) * (3 * QF);
  // warpgroup 0: x face j, i+1/2 from cells i-1 .. i+2 of row j; warpgroup
  // 1: y face j+1/2 from rows j-1 .. j+2 of column i, in the rotated frame
  // (one code path for both: the stencil pointers and the swap differ)
  const bool yf = wg != 0;
  const float* p0 = yf ? qring + ((tau + 1) % 5) * (3 * QF) + m + 2 : qj + m + 1;
  const float* p1 = qj + m + 2;
  const float* p2 = yf ? qring + ((tau + 3) % 5) * (3 * QF) + m + 2 : qj + m + 3;
  const float* p3 = yf ? qring + ((tau + 4) % 5) * (3 * QF) + m + 2 : qj + m + 4;
  float qm[3], q0[3], q1[3], qp[3], L[3], R[3], F[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    qm[c] = p0[c * QF];
    q0[c] = p1[c * QF];
    q1[c] = p2[c * QF];
    qp[c] = p3[c * QF];
  }
  learned_face(qm, q0, q1, qp, wd, Q.hmin, L, R);
  float f1, f2;
  hll_swe<float>(L[0], yf ? L[2] : L[1], yf ? L[1] : L[2], R[0], yf ? R[2] : R[1], yf ? R[1] : R[2], a.g,
                 F[0], f1, f2);
  F[1] = yf ? f2 : f1;
  F[2] = yf ? f1 : f2;
  if (!yf) {
    float* Fs = Fb + (tau & 1) * (F_SLOT / 4);
#pragma unroll
    for (int c = 0; c < 3; ++c) Fs[c * (W + 1) + m + 1] = F[c];
    if (m == W - 1) {
      float* fo = reinterpret_cast<float*>(sbuf + OFF_FXO) + (Q.nt & 1) * 4;
      *reinterpret_cast<float4*>(fo) = make_float4(F[0], F[1], F[2], 0.f);
      tc::fence_proxy_async_smem();
      copy_to_cta(sbuf + OFF_FXI + (Q.nt & 1) * 16, fo, 16, tick_done, X.east);
    }
  } else {
    float* Gs = Gb + (tau % 3) * (G_SLOT / 4);
#pragma unroll
    for (int c = 0; c < 3; ++c) Gs[c * W + m] = F[c];
  }
}

// Wait for phase `parity` of `mbar` by polling without suspending (for the
// issuing warp, whose waits are short and on the critical path); gives up
// after `max_iters` polls and returns false.
__device__ __forceinline__ bool mbar_spin_bounded(uint64_t* mbar, uint32_t parity, uint32_t max_iters) {
  for (uint32_t i = 0; i < max_iters; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tc::smem_u32(mbar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Per-warp arrival on a local mbarrier: the warp's lanes first order their
// shared-memory and TMEM accesses, then lane 0 arrives (release).
__device__ __forceinline__ void warp_arrive(uint64_t* mbar, uint32_t tx, bool with_tx) {
  tc::fence_before_sync();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    if (with_tx) mbar_arrive_expect_tx(mbar, tx);
    else mbar_arrive(mbar);
  }
}

// The staging warps' part of tick Q.tau (warps 1-3 of warpgroup 2): once
// the tick's MMAs have read the slot, the layer-1 input of row t+1 from the
// raw row and, if `early_ready`, the "inputs ready" arrival; then the FP32
// state row t-4 into the ring and the raw row t+2 of the next tick
// (cp.async, landed before the "done" arrival), and an L2 prefetch of row
// t+3.  `prev_done`: tick nt - 1 of the stream done (null for the first tick).
// Called by every staging thread each phase, `ok` or not (the named barrier
// must see all 96); returns `ok` and the outcome of its waits.
template <int STAGE>
__device__ __forceinline__ bool staging(Stream& Q, uint8_t* sbuf, uint64_t* mma, uint64_t* ready,
                                        uint64_t* prev_done, uint32_t prev_parity, const Args& a,
                                        const Ctx& X, bool ok, bool early_ready) {
  const int tau = Q.tau, t = Q.u0 - 3 + tau;
  const int k = X.m - 32, n = W - 32;
  const float* qb = a.qin + (long long)Q.b * a.member;
  float* raw = reinterpret_cast<float*>(sbuf + OFF_RAW);
  // every read of the previous tick is done, its rows are staged
  if (ok && prev_done) ok = tc::mbar_wait_bounded(prev_done, prev_parity, WAIT_ITERS);
  if (ok) ok = tc::mbar_wait_bounded(mma, Q.parity, WAIT_ITERS);
  if (ok && tau + 1 < Q.ntau) build_l1_row(sbuf + OFF_L1 + (tau % 3) * L1_SLOT, raw, a, k, n);
  tc::fence_proxy_async_smem();
  if (early_ready) warp_arrive(ready, 0, false);
  asm volatile("bar.sync 5, 96;" ::: "memory");          // every read of the raw row is done
  if (ok) {
    load_q_row(reinterpret_cast<float*>(sbuf + OFF_Q) + (tau % 5) * (3 * QF), a, qb, t - 4, X.X0, k, n);
    if (tau + 2 < Q.ntau) fetch_raw_row(raw, a, qb, t + 2, X.X0, k);
    if (tau + 3 < Q.ntau) prefetch_row(a, qb, t + 3, X.X0, k);
    asm volatile("cp.async.wait_all;\n" ::: "memory");  // the rows have landed
  }
  return ok;
}

// Max / or over the four warps of draining warpgroup 0 (named barrier 3);
// the result is in thread 0.
__device__ __forceinline__ void wg0_reduce_max_or(float& m, unsigned& bad, unsigned* red) {
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[w] = __float_as_uint(m);
    red[4 + w] = bad;
  }
  asm volatile("bar.sync 3, 128;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int i = 1; i < 4; ++i) {
      m = fmaxf(m, __uint_as_float(red[i]));
      bad |= red[4 + i];
    }
  }
}

// One phase: the tick of stream M (index ms) on the tensor core, the
// epilogue of stream E (index ms ^ 1, whose MMAs were issued in the previous
// phase) on the CUDA cores.  The stream indices are run-time values so that
// the kernel holds one copy of the phase code.
//
// Hand-offs (all mbarriers, per stream s):
//  * mma[s]: the tick's MMAs have completed, in this CTA and in the
//    neighbours whose halos they read (multicast commit);
//  * ready[s]: the inputs of the stream's next tick are in place: the hidden
//    rows and the slot move (8 draining warps), the layer-1 input row (3
//    staging warps; warp 10 once it has also placed the neighbours' halo
//    columns, which arrive on halo_in[s] as 384 bytes of copies);
//  * done[s][n & 1]: tick n is complete (draining and staging warps, and the
//    16-byte east-face flux from the west neighbour); tick n + 1 waits for it
//    before it reads the staged rows and fluxes or overwrites their slots.
// The issuing thread waits only for ready[M]; the other warps wait for
// mma[E] and done[E] of the previous tick, both normally complete long before.
template <int STAGE>
__device__ __forceinline__ void phase(Stream& M, Stream& E, const Args& a, Ctx& X, int ms) {
  const int es = ms ^ 1;
  if (M.active) M.pending = true;      // its MMAs go to the tensor core in this phase
  if (E.pending) {
    uint8_t* sbuf = X.smem + OFF_STREAMS + es * STREAM_BYTES;
    uint64_t* ready = &X.mbar[2 + es];
    uint64_t* done = &X.mbar[4 + 2 * es + (E.nt & 1)];
    uint64_t* prev_done = E.nt ? &X.mbar[4 + 2 * es + ((E.nt - 1) & 1)] : nullptr;
    const uint32_t prev_parity = ((E.nt - 1) >> 1) & 1;
    // at the end of a segment the next segment's first layer-1 rows are
    // written below; the "inputs ready" arrivals wait for them
    const bool seg_end = E.tau + 1 == E.ntau;
    bool ok = !X.failed;
    if (X.wg < 2) {
      const uint32_t tm = X.tmem + 256u * es + X.lane_off;
      // the previous tick's fluxes and staged rows (normally long complete):
      // warpgroup 0 updates row t-8 while the MMAs run
      if (ok && prev_done) ok = tc::mbar_wait_bounded(prev_done, prev_parity, WAIT_ITERS);
      if (ok && X.wg == 0) update_cell<STAGE>(E, sbuf, a, X, X.m);
      if (ok) ok = tc::mbar_wait_bounded(&X.mbar[es], E.parity, WAIT_ITERS);
      tc::fence_after_sync();
      float wd[18];
      if (ok) drain_rows(E, sbuf, tm, X);
      // every draining warp has written its rows and halo columns: lanes 0
      // and 1 send the halos
      asm volatile("bar.sync 2, %0;" ::"n"(EPI_THREADS) : "memory");
      if (ok && X.tid < 2) send_halos(sbuf, &X.mbar[8 + es], X);
      const uint32_t ring_slot = tm + ACC4 + R4 * (E.nt % 3u);
      if (ok) drain_coeffs(ring_slot, X.bias + 3 * snk::HID, X.wg, wd);
      asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");   // slot-0 reads of both warpgroups done
      if (ok) move_slots(tm, ring_slot, X.wg);
      if (!seg_end) warp_arrive(ready, 0, false);
      if (ok) epilogue_faces(E, sbuf, a, X, done, wd);
      warp_arrive(done, 0, false);
    } else if (X.m >= 32) {
      const bool halo_warp = X.m >= 64 && X.m < 96;   // warp 10
      ok = staging<STAGE>(E, sbuf, &X.mbar[es], ready, prev_done, prev_parity, a, X, ok,
                          !seg_end && !halo_warp);
      warp_arrive(done, 16, X.m < 64);
      if (halo_warp) {
        // every tick, so that the halo barrier's phases stay in step
        ok = place_halos(E, sbuf, &X.mbar[8 + es], ok);
        if (!seg_end) warp_arrive(ready, 0, false);
      }
    }
    if (!ok && !X.failed) {
      X.failed = true;
      atomicOr(a.err, 1u);
    }
    E.parity ^= 1u;
    E.pending = false;
    ++E.nt;
    if (++E.tau == E.ntau) {
      // segment done: close the member's stage-2 reduction, start the next segment
      if (STAGE == 2 && X.wg == 0) {
        // draining warpgroup 0 holds the Courant rates of the rows it updated
        float mx = E.amax;
        unsigned bd = E.bad;
        wg0_reduce_max_or(mx, bd, X.red);
        if (X.tid == 0) {
          const long long R = a.rows, Sn = a.nstreams;
          const long long first = stream_of_row((long long)E.b * a.ny, R, Sn);
          const long long last = stream_of_row((long long)(E.b + 1) * a.ny - 1, R, Sn);
          publish_and_close(a.ctrl + E.b, a.dp, mx, bd, (unsigned)(a.cs * (last - first + 1)), true);
        }
      }
      E.active = next_segment(E, a, X.crank);
      if (E.active) {
        segment_prologue(E, sbuf, a, X.X0, X.m, X.wg, !X.failed);
        tc::fence_proxy_async_smem();
      }
      if (X.wg < 2) warp_arrive(ready, 0, false);
      else if (X.m >= 32) warp_arrive(ready, 0, false);
    }
  }
}

// One phase of the issuing warp: the same stream states as the other warps,
// reduced to what the MMA issue needs (the tick's slots, the "inputs ready"
// phase to wait for, segment changes); lane 0 issues the MMAs.
// Returns false once both streams are done.
__device__ __forceinline__ bool issuer_phase(Stream& M, Stream& E, const Args& a, Ctx& X, int ms) {
  if (!(M.active || E.active || M.pending || E.pending)) return false;
  const int lane = threadIdx.x & 31;
  if (M.active) {
    if (!X.failed) {
      bool ok = M.nt == 0 || mbar_spin_bounded(&X.mbar[2 + ms], (M.nt - 1) & 1, 64u * WAIT_ITERS);
      ok = __all_sync(0xffffffffu, ok);
      if (ok) {
        if (lane == 0) {
          tc::fence_after_sync();
          Descs D = X.D;
          if (ms) {
            D.a_l1 = dplus(D.a_l1, STREAM_BYTES);
            D.a_in = dplus(D.a_in, STREAM_BYTES);
          }
          issue_tick(D, X.tmem + 256u * ms, M.tau, M.nt, &X.mbar[ms], X.commit_mask);
        }
        __syncwarp();
      } else {
        X.failed = true;
        if (lane == 0) atomicOr(a.err, 1u);
      }
    }
    M.pending = true;
  }
  if (E.pending) {
    E.pending = false;
    ++E.nt;
    if (++E.tau == E.ntau) E.active = next_segment(E, a, X.crank);
  }
  return true;
}

// The issuing warp's loop, two phases per iteration (the streams' roles
// alternate without copying their states).
__device__ __forceinline__ void issuer_loop(Stream S0, Stream S1, const Args& a, Ctx& X) {
#pragma unroll 1
  for (;;) {
    if (!issuer_phase(S0, S1, a, X, 0)) break;
    if (!issuer_phase(S1, S0, a, X, 1)) break;
  }
}

template <int STAGE>
__global__ void __launch_bounds__(NT, 1) learned_fused_kernel(Args a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  float* bias = reinterpret_cast<float*>(smem + OFF_BIAS);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + OFF_TSLOT);

  Ctx X;
  X.smem = smem;
  X.bias = bias;
  X.mbar = reinterpret_cast<uint64_t*>(smem + OFF_MBAR);
  X.red = reinterpret_cast<unsigned*>(smem + OFF_RED);
  X.tid = threadIdx.x;
  X.m = X.tid & (W - 1);                  // TMEM lane = column within the CTA
  X.wg = X.tid >> 7;                      // 0, 1: drain TMEM; 2: update and stage
  X.issuer = X.tid == EPI_THREADS;        // first lane of warpgroup 2
  X.failed = false;
  X.lane_off = (uint32_t)(32 * ((X.tid >> 5) & 3)) << 16;
  X.crank = cluster_rank();
  X.X0 = (int)X.crank * W;
  X.west = (X.crank + a.cs - 1) % a.cs;
  X.east = (X.crank + 1) % a.cs;
  X.commit_mask = (uint16_t)((1u << X.crank) | (1u << X.west) | (1u << X.east));
  const long long cluster = blockIdx.x / a.cs;

  if ((X.tid >> 5) == ISSUE_WARP) {
    tc::tmem_alloc(tslot, TCOLS);         // the issuing warp owns the TMEM allocation
    if (X.issuer) {
      // one arrival per tick from this CTA and from each distinct neighbour
      const uint32_t arrivals = (uint32_t)__popc((unsigned)X.commit_mask);
      tc::mbar_init(&X.mbar[0], arrivals);
      tc::mbar_init(&X.mbar[1], arrivals);
      // ready and done: one arrival per draining and per staging warp
      for (int i = 2; i < 8; ++i) tc::mbar_init(&X.mbar[i], EPI_THREADS / 32 + 3);
      // halos: one local arrival (with the expected bytes) per tick
      tc::mbar_init(&X.mbar[8], 1);
      tc::mbar_init(&X.mbar[9], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  // weights and biases
  for (int i = X.tid; i < W1_BYTES / 16; i += NT) cp_async16(smem + OFF_W1 + i * 16, a.w1g + i * 8);
  for (int i = X.tid; i < WH_BYTES / 16; i += NT) {
    cp_async16(smem + OFF_W2 + i * 16, a.w2 + i * 8);
    cp_async16(smem + OFF_W3 + i * 16, a.w3 + i * 8);
  }
  for (int i = X.tid; i < W4_BYTES / 16; i += NT) cp_async16(smem + OFF_W4 + i * 16, a.w4 + i * 8);
  for (int i = X.tid; i < N_BIAS; i += NT) {
    if (i < 3 * snk::HID) {
      bias[i] = a.params[a.bias_off[i / snk::HID] + i % snk::HID];
    } else {
      // layer 4: b[3 s + j] - b[3 s + 2] for difference 2 s + j
      const int d = i - 3 * snk::HID, st = d / 2, jj = d % 2;
      bias[i] = a.params[a.bias_off[3] + 3 * st + jj] - a.params[a.bias_off[3] + 3 * st + 2];
    }
  }

  // the two streams of this cluster and their first segments
  Stream S0, S1;
  S0.g = (2 * cluster) * a.rows / a.nstreams;
  S0.g_end = (2 * cluster + 1) * a.rows / a.nstreams;
  S1.g = S0.g_end;
  S1.g_end = (2 * cluster + 2) * a.rows / a.nstreams;
  S0.parity = S1.parity = 0u;
  S0.nt = S1.nt = 0u;
  S0.pending = S1.pending = false;
  S0.active = next_segment(S0, a, X.crank);
  S1.active = next_segment(S1, a, X.crank);
  if (S0.active) segment_prologue(S0, smem + OFF_STREAMS, a, X.X0, X.m, X.wg, true);
  if (S1.active) segment_prologue(S1, smem + OFF_STREAMS + STREAM_BYTES, a, X.X0, X.m, X.wg, true);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  X.tmem = *tslot;
  const uint32_t sb = tc::smem_u32(smem);
  X.D.a_l1 = tc::sdesc(sb + OFF_STREAMS + OFF_L1, W * 16, 128);
  X.D.a_in = tc::sdesc(sb + OFF_STREAMS + OFF_IN, FP * 16, 128);
  X.D.b_w1 = tc::sdesc(sb + OFF_W1, snk::HID * 16, 128);
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    constexpr uint32_t N = snk::HID;
    const uint32_t wl = sb + (l == 0 ? OFF_W2 : OFF_W3);
    X.D.b_ky0[l] = tc::sdesc(wl, N * 16, 128);
    X.D.b_pair[l] = tc::sdesc(wl + 3 * snk::CG_HID * N * 16, 2 * N * 16, 128);
  }
  X.D.b_ring = tc::sdesc(sb + OFF_W4, snk::W4R_ROWS * 16, 128);
  if (X.wg < 2) {
    // layer 4's ring slots start cleared (its MMAs only accumulate):
    // warpgroup 0 columns 0-39, warpgroup 1 40-79 of each stream's ring
    const float z16[16] = {};
    const float z8[8] = {};
#pragma unroll
    for (int st = 0; st < 2; ++st) {
      const uint32_t base = X.tmem + 256u * st + X.lane_off + ACC4 + 40u * X.wg;
      tmem_st16(base, z16);
      tmem_st16(base + 16, z16);
      tmem_st8(base + 32, z8);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    tc::fence_before_sync();
  }
  // every CTA of the cluster is running (and its mbarriers initialised)
  // before any remote store or multicast arrival
  cluster_arrive();
  cluster_wait();

  if ((X.tid >> 5) == ISSUE_WARP) {
    issuer_loop(S0, S1, a, X);
  } else {
    // M: the stream whose tick goes to the tensor core in this phase (index
    // ms), E: the other one; they swap roles every phase
    Stream M = S0, E = S1;
    int ms = 0;
#pragma unroll 1
    for (;;) {
      if (!(M.active || E.active || M.pending || E.pending)) break;
      phase<STAGE>(M, E, a, X, ms);
      const Stream T = M;
      M = E;
      E = T;
      ms ^= 1;
    }
    // The last tick of each stream: its "inputs ready" and "done" phases
    // still receive the neighbours' copies; wait until they have landed.  No
    // MMA is in flight unless a wait gave up; give those a bounded wait too.
    if (X.tid == 0) {
      const uint32_t nts[2] = {ms ? E.nt : M.nt, ms ? M.nt : E.nt};
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (nts[s]) {
          tc::mbar_wait_bounded(&X.mbar[2 + s], (nts[s] - 1) & 1, WAIT_ITERS);
          tc::mbar_wait_bounded(&X.mbar[4 + 2 * s + ((nts[s] - 1) & 1)], ((nts[s] - 1) >> 1) & 1, WAIT_ITERS);
        }
      }
    }
    if (X.failed) {
      tc::mbar_wait_bounded(&X.mbar[ms], M.parity, WAIT_ITERS);
      tc::mbar_wait_bounded(&X.mbar[ms ^ 1], E.parity, WAIT_ITERS);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  // no CTA leaves while a neighbour may still address its shared memory
  cluster_arrive();
  cluster_wait();
  if ((X.tid >> 5) == ISSUE_WARP) tc::tmem_dealloc(X.tmem, TCOLS);
}

}  // namespace fused

bool learned_fused_supported(int nx, int ny) {
  return nx % fused::W == 0 && nx / fused::W <= fused::MAX_CS && ny >= 1;
}
// (A subdomain ring in x would shift the 128-column tiles off the grid's
// columns; the fused kernel takes rings of rows only.)

namespace {

template <int STAGE>
cudaError_t launch_fused_stage(const fused::Args& a, cudaStream_t s) {
  using namespace fused;
  auto kern = learned_fused_kernel<STAGE>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // clusters that fit on the device at once (one CTA per SM), cached per size
  static int max_clusters[MAX_CS + 1] = {};
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)a.cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (!max_clusters[a.cs]) {
    int n = 0;
    cfg.gridDim = dim3((unsigned)a.cs);
    cudaError_t e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    max_clusters[a.cs] = n;
  }
  // every stream gets at least one row (with a single row in total, the
  // first stream of the only cluster stays empty)
  long long clusters = max_clusters[a.cs];
  if (clusters > a.rows / 2) clusters = a.rows / 2 > 0 ? a.rows / 2 : 1;
  fused::Args args = a;
  args.nstreams = 2 * clusters;
  cfg.gridDim = dim3((unsigned)(clusters * a.cs));
  return cudaLaunchKernelEx(&cfg, kern, args);
}

}  // namespace

cudaError_t launch_learned_fused(const Geom& g, int stage, const float* qin, const float* qn,
                                 float* qout, const snk::Net& net, const float* hmin, Ctrl* ctrl,
                                 const DtParams* dp, cudaStream_t s) {
  if (!learned_fused_supported(g.nx, g.ny)) return cudaErrorInvalidValue;
  const snk::ParamLayout L = snk::param_layout();
  fused::Args a{};
  a.qin = qin;
  a.qn = qn;
  a.qout = qout;
  a.w1g = net.w1g;
  a.w2 = net.wpair[1];
  a.w3 = net.wpair[2];
  a.w4 = net.w4ring;
  a.params = net.params;
  for (int l = 0; l < 4; ++l) a.bias_off[l] = L.b[l];
  for (int c = 0; c < 3; ++c) {
    a.mean[c] = net.mean[c];
    a.rstd[c] = 1.f / net.std_[c];
  }
  a.hmin = hmin;
  a.ctrl = ctrl;
  a.dp = dp;
  a.nx = g.nx;
  a.ny = g.ny;
  a.cs = g.nx / fused::W;
  a.plane = g.plane();
  a.member = g.member();
  a.rows = (long long)g.B * g.ny;
  a.rdx = (float)(1.0 / g.dx);
  a.rdy = (float)(1.0 / g.dy);
  a.g = g.phys;
  a.err = net.err;
  a.hy = g.hy;
  return stage == 1 ? launch_fused_stage<1>(a, s) : launch_fused_stage<2>(a, s);
}

}  // namespace fvk
