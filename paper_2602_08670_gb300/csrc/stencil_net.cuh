// stencil_net.cuh — the learned-stencil CNN (internal interface).
//
// Section 2.5.3, fourth approach: a CNN maps the cell-average state to
// constrained reconstruction coefficients.  Architecture: x = (q - mean)/std
// per channel; four 3x3 convolutions with periodic padding, 3 -> 32 -> 32 ->
// 32 -> 36 channels, ReLU after the first three.  The 36 outputs of a cell are
// 2 directions x 3 variables x 2 sides x 3 taps; each 3-tap stencil is
// normalised to w = e_centre + r - mean(r) (weights sum to one; r = 0 is the
// first-order scheme).
//
// Section 2.5.3, third approach (NET_FACE): the same backbone with GeLU in
// place of ReLU and 12 outputs per cell, the states on its four sides
// (west, east, south, north) x (h, hu, hv) at channel 3 side + var; the
// depths pass through Softplus, the momenta are de-normalised
// (mean + std r).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fv.h"

namespace snk {

constexpr int C_IN = 3;
constexpr int HID = 32;
constexpr int N_OUT = 36;
constexpr int N_OUT_PAD = 48;        // MMA N must be a multiple of 16
constexpr int N_PARAMS = 29796;      // W1 b1 W2 b2 W3 b3 W4 b4 (PyTorch order)
constexpr int CG_IN0 = 2;            // layer-1 input: 3 channels padded to 16 (2 groups of 8)
constexpr int CG_HID = 4;            // 32 channels = 4 groups of 8
constexpr int TILE = 128;            // cells per MMA tile (M)
enum { NET_STENCIL = 0, NET_FACE = 1 };
constexpr int N_OUT_FACE = 12;       // 4 sides x 3 variables
constexpr int N_OUT_FACE_PAD = 16;
constexpr int N_PARAMS_FACE = 22860; // W1 b1 W2 b2 W3 b3 W4[12] b4[12]

// Offsets of each layer's weight and bias in the flat parameter vector.
struct ParamLayout {
  int w[4], b[4], cout[4], cin[4];
};
ParamLayout param_layout(int kind = NET_STENCIL);
int n_params(int kind);

// Device buffers of one network.
struct Net {
  int kind = NET_STENCIL;      // NET_STENCIL (fourth approach) or NET_FACE (third)
  float* params = nullptr;     // FP32 master parameters [n_params(kind)]
  uint16_t* wf[4] = {};        // forward B operands, BF16 [9][CG_in][N][8]
  uint16_t* wb[4] = {};        // backward (dX) B operands, BF16 [9][CG_out][N_in][8] (layer 1:
                               // N_in = DQ_N, the 3 state channels padded)
  uint16_t* w1g = nullptr;     // layer 1 with the three x taps gathered into K, BF16
                               // [ky][2][HID][8]: channel c = 3 kx + var (c < 9, rest 0)
  uint16_t* wpair[3] = {};     // layers 2..3 for the row-pipelined kernel, BF16: the taps
                               // ky = 0 as [kx][4][N][8], then ky = 2 and ky = 1 stacked
                               // along N as [kx][4][2N][8] (rows n < N: ky = 2)
  uint16_t* w4ring = nullptr;  // layer 4 for the row-pipelined kernel, BF16 [kx][4][128][8]:
                               // per 3-tap stencil s (12 of them, output channels 3 s + j)
                               // the differences W[3 s] - W[3 s + 2], W[3 s + 1] - W[3 s + 2]
                               // (rows 2 s, 2 s + 1 of a 24-row block), blocks of the taps
                               // ky = 2, 1, 0, 2, 1 (rows 0..119), rows 120..127 zero
  float mean[3] = {0, 0, 0};
  float std_[3] = {1, 1, 1};
  unsigned* err = nullptr;     // device error word (bounded waits that gave up)
};

// Per-call activation workspace for `cells` = B * plane cells.
struct Acts {
  uint16_t* a[3] = {};         // post-activation outputs of layers 1..3, BF16 [B][4][plane][8]
  uint16_t* z[3] = {};         // face-state training only: pre-activations, BF16 [B][4][plane][8]
  long long cells = 0;
};

bool grid_supported(int nx);   // nx % 128 == 0, or nx in {8, 16, 32, 64}
constexpr int W1G_ELEMS = 3 * 2 * HID * 8;
constexpr int DQ_N = 16;             // N of the first layer's dX convolution (3 channels padded)
constexpr int W4R_BLOCK = 24;        // rows of one tap in w4ring: 12 stencils x 2 differences
constexpr int W4R_ROWS = 128;        // 5 tap blocks + 8 zero rows
constexpr int W4R_ELEMS = 3 * CG_HID * W4R_ROWS * 8;

// Pack the FP32 master parameters into the BF16 MMA operand layouts.
cudaError_t repack(Net& net, cudaStream_t s);

// Forward of the whole network on q [B][3][ny][nx] (FP32, device).  Writes
// the normalised weights w [B][36][ny][nx] (FP32) and keeps the hidden
// activations in `acts` (which must hold B*ny*nx cells).  If raw != nullptr
// the un-normalised outputs r [B][36][ny][nx] are written instead of w.
cudaError_t forward(const Net& net, const float* q, int B, int ny, int nx, Acts& acts, float* w,
                    float* raw, cudaStream_t s);

// Forward of a NET_FACE network: the side states [B][12][ny][nx] (FP32) into
// `sides`, or, if raw != nullptr, the un-activated outputs r there instead.
cudaError_t forward_faces(const Net& net, const float* q, int B, int ny, int nx, Acts& acts,
                          float* sides, float* raw, cudaStream_t s);

// with_z: also the pre-activation buffers (backward of the face-state network).
cudaError_t acts_reserve(Acts& acts, long long cells, bool with_z = false);
void acts_free(Acts& acts);

// Backward workspace.
struct Grads {
  uint16_t* dr = nullptr;       // cotangent of the raw outputs, BF16 [B][6][plane][8]
  uint16_t* da[2] = {};         // cotangents of hidden pre-activations, BF16 [B][4][plane][8]
  float* part = nullptr;        // weight-gradient partial sums (two buffers, alternate layers)
  float* part2 = nullptr;
  long long cells = 0, part_floats = 0;
  static constexpr int NEV = 9;
  cudaStream_t aux = nullptr;   // the weight gradients run here, beside the dX convolutions
  cudaStream_t red = nullptr;   // their partial-sum reductions
  cudaEvent_t ev[NEV] = {};     // fork / join points between the streams
};
long long backward_partials_floats(int B, int ny, int nx);
cudaError_t backward_reserve(Grads& g, long long cells, long long partial_floats);
void backward_free(Grads& g);

// Vector-Jacobian product of forward() at q given the cotangent dw of the
// normalised coefficients [B][36][ny][nx]: adds scale * (d params) to
// dparams [N_PARAMS] and, if dq != nullptr, the cotangent of q to dq
// [B][3][ny][nx] (scale applies to dparams only).  `acts` must hold the
// activations forward() produced for this q.  Cotangents between layers are
// BF16 (tensor-core operands); weight gradients accumulate in FP32.
cudaError_t backward(const Net& net, const float* q, int B, int ny, int nx, const Acts& acts,
                     const float* dw, float* dq, float* dparams, float scale, Grads& g,
                     cudaStream_t s);
// The same from the cotangent of the raw network outputs, already in g.dr
// (BF16 [B][6][plane][8], the normalisation's VJP applied).
cudaError_t backward_from_raw(const Net& net, const float* q, int B, int ny, int nx, const Acts& acts,
                              float* dq, float* dparams, float scale, Grads& g, cudaStream_t s);

// The same for a NET_FACE network: ds is the cotangent of the side states
// [B][12][ny][nx], `sides` the side states forward_faces() produced for this
// q, and `acts` must hold its activations and pre-activations (with_z).
cudaError_t backward_faces(const Net& net, const float* q, int B, int ny, int nx, const Acts& acts,
                           const float* sides, const float* ds, float* dq, float* dparams, float scale,
                           Grads& g, cudaStream_t s);

}  // namespace snk

struct fv_net {
  snk::Net n;
  snk::Acts ws;                 // workspace of stencil_net_forward / _backward
  snk::Grads bw;                // workspace of stencil_net_backward / face_net_backward
  float* scratch = nullptr;     // forward outputs recomputed by the backward calls
  long long scratch_floats = 0;
  float* adam_m = nullptr;      // Adam moments (stencil_net_adam_step)
  float* adam_v = nullptr;
  cudaStream_t stream = nullptr;
};
