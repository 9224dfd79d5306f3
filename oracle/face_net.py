"""FP64 oracle of the face-state CNN variant (test infrastructure only).

Section 2.5.3, the third approach (a CNN computes the boundary states
directly; results in Section 5.3): a CNN maps the cell averages of a cell's
neighbourhood to the states on its four sides, Q^l, Q^r, Q^b, Q^u; each face
flux pairs the two states that meet there, and the flux, divergence and
SSP-RK2 of the plain scheme follow.  Section 5.3 trains it with the solver in
the loss (the rollout loss of Eq. 2.28).

Readings where the paper is silent or loose (each listed with its reason in
the design notes):
  * Network: x = (q - mean) / std per variable (the same normalisation as
    the fourth approach); four 3x3 convolutions with circular padding,
    3 -> 32 -> 32 -> 32 -> 12 channels, GeLU (the erf form) after the first
    three, the last one linear.
  * 12 outputs per cell: side s in (l, r, b, u) = (west, east, south,
    north), variable v in (h, hu, hv), channel 3 s + v.  The depth outputs
    pass through Softplus (so every reconstructed depth is positive and no
    fallback is needed): h_side = softplus(r).  The momentum outputs are
    de-normalised: m_side = mean_v + std_v r.
  * The flux through the face between cells i-1 and i is the HLL flux of
    Q^r_{i-1} (left state) and Q^l_i (right state); in y, of Q^u_{j-1} and
    Q^b_j, in the rotated frame of Eq. 2.24.  The thesis's remark that the
    fluxes of a shared side are equal and opposite is the conservative
    update (each face flux enters both cells).
  * The CNN runs at every Runge-Kutta stage; dt follows the CFL rule of the
    plain scheme (Eq. 2.10) on the stage-free state.

Precision mirror: with ``round_bf16=True`` the network input and every hidden
activation are rounded to bfloat16 and the weights are expected to be
bfloat16 values, as on the GPU; sums stay FP64.  ``run(..., dtype=float32)``
replays the same algorithm in single precision (sums, GeLU, the flux and
the update): its distance from the FP64 run is the roundoff yardstick of the
GPU parity tests.  Because the depth outputs feed the pressure flux
directly, a BF16 rounding of a hidden activation that flips between the two
precisions moves the momentum by far more than FP32 roundoff alone.
"""
from __future__ import annotations

import dataclasses

import torch

from . import fv
from .stencil_net import bf16, conv3x3_periodic, f32

C_SWE = 3
HIDDEN = 32
N_OUT = 12           # 4 sides x 3 variables
LAYER_SHAPES = [(HIDDEN, C_SWE), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (N_OUT, HIDDEN)]
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3


def out_channel(side: int, var: int) -> int:
    """Index of one output among the 12 of a cell."""
    return 3 * side + var


def n_params() -> int:
    return sum(co * ci * 9 + co for co, ci in LAYER_SHAPES)


@dataclasses.dataclass
class FaceNetParams:
    W: list            # 4 tensors [Cout][Cin][3][3]
    b: list            # 4 tensors [Cout]
    mean: torch.Tensor  # [3]
    std: torch.Tensor   # [3]

    @staticmethod
    def from_flat(flat: torch.Tensor, mean, std) -> "FaceNetParams":
        """Unpack the flat parameter vector: W1, b1, W2, b2, W3, b3, W4, b4
        (PyTorch Conv2d layout)."""
        W, b, off = [], [], 0
        for co, ci in LAYER_SHAPES:
            n = co * ci * 9
            W.append(flat[off:off + n].reshape(co, ci, 3, 3))
            off += n
            b.append(flat[off:off + co])
            off += co
        return FaceNetParams(W, b, torch.as_tensor(mean, dtype=torch.float64),
                             torch.as_tensor(std, dtype=torch.float64))

    def flat(self) -> torch.Tensor:
        parts = []
        for W, b in zip(self.W, self.b):
            parts += [W.reshape(-1), b.reshape(-1)]
        return torch.cat(parts)


def gelu(x: torch.Tensor) -> torch.Tensor:
    """GeLU, x Phi(x) with Phi the standard normal distribution function,
    written through the error function: Phi(x) = (1 + erf(x / sqrt 2)) / 2."""
    return 0.5 * x * (1.0 + torch.erf(x * 0.7071067811865476))


def softplus(x: torch.Tensor) -> torch.Tensor:
    """log(1 + e^x), evaluated as log(e^0 + e^x) without overflow."""
    return torch.logaddexp(torch.zeros_like(x), x)


def _round_bf16(x: torch.Tensor) -> torch.Tensor:
    """Round to bfloat16 (nearest-even), in the precision of x; the FP64
    path keeps the graph through the rounding."""
    if x.dtype == torch.float64:
        return bf16(x)
    return x.to(torch.bfloat16).to(x.dtype)


def net_raw(q: torch.Tensor, p: FaceNetParams, round_bf16: bool = True) -> torch.Tensor:
    """Raw network output r[B][12][ny][nx] for the state q (SWE), computed
    in the precision of q."""
    dt_ = q.dtype
    x = (q - p.mean.to(dt_).view(1, -1, 1, 1)) / p.std.to(dt_).view(1, -1, 1, 1)
    if round_bf16:
        x = _round_bf16(x)
    for layer in range(4):
        x = conv3x3_periodic(x, p.W[layer].to(dt_), p.b[layer].to(dt_))
        if layer < 3:
            x = gelu(x)
            if round_bf16:
                x = _round_bf16(x)
    return x


def side_states(raw: torch.Tensor, p: FaceNetParams) -> torch.Tensor:
    """The 12 side states [B][4][3][ny][nx] (side, variable) from the raw
    outputs: Softplus on the depths, de-normalised momenta."""
    B, _, ny, nx = raw.shape
    r = raw.reshape(B, 4, 3, ny, nx)
    mean, std = p.mean.to(raw.dtype), p.std.to(raw.dtype)
    h = softplus(r[:, :, 0])
    hu = mean[1] + std[1] * r[:, :, 1]
    hv = mean[2] + std[2] * r[:, :, 2]
    return torch.stack([h, hu, hv], dim=2)


def face_rhs(q: torch.Tensor, sides: torch.Tensor, dx: float, dy: float, g: float = 9.81) -> torch.Tensor:
    """L(q) from the side states [B][4][3][ny][nx]: the face i+1/2 (stored at
    index i) pairs Q^r_i with Q^l_{i+1}; j+1/2 pairs Q^u_j with Q^b_{j+1}."""
    QLx = sides[:, EAST]
    QRx = torch.roll(sides[:, WEST], -1, dims=-1)
    Fx = fv.face_flux(QLx, QRx, *fv.X_FACE, fv.SWE, g, 1.4)
    QLy = sides[:, NORTH]
    QRy = torch.roll(sides[:, SOUTH], -1, dims=-2)
    Gy = fv.face_flux(QLy, QRy, *fv.Y_FACE, fv.SWE, g, 1.4)
    return fv.divergence_update(Fx, Gy, dx, dy)


def rhs(q, p: FaceNetParams, dx, dy, g=9.81, round_bf16=True):
    return face_rhs(q, side_states(net_raw(q, p, round_bf16), p), dx, dy, g)


def step(q, p: FaceNetParams, dt, g=9.81, round_bf16=True):
    dx, dy = fv.grid_spacing(q)
    return fv.ssp_rk2(q, dt, lambda s: rhs(s, p, dx, dy, g, round_bf16))


def run(q0, p: FaceNetParams, nsteps: int, *, cfl: float = 0.5, dt_mode: str = fv.DT_ADAPTIVE,
        dt_fixed=None, dts=None, g: float = 9.81, round_bf16: bool = True, dtype=torch.float64):
    """``nsteps`` steps; dt by the CFL rule (Eq. 2.10) of the state at the
    start of each step, fixed, or replayed.  Returns (q, t, dt_history).
    ``dtype`` float32 replays the algorithm in single precision."""
    q = torch.as_tensor(q0).to(dtype).clone()
    B = q.shape[0]
    dx, dy = fv.grid_spacing(q)
    t = torch.zeros(B, dtype=dtype)
    hist = []
    for n in range(nsteps):
        if dt_mode == fv.DT_ADAPTIVE:
            dt = fv.cfl_dt(q, fv.SWE, cfl, dx, dy, g).to(dtype)
        elif dt_mode == fv.DT_FIXED:
            dt = torch.full((B,), float(dt_fixed), dtype=dtype)
        else:
            d = torch.as_tensor(dts[n]).to(dtype)
            dt = d.expand(B).clone() if d.dim() == 0 else d.clone()
        q = step(q, p, dt.view(B, 1, 1, 1), g, round_bf16)
        t = t + dt
        hist.append(dt)
    dt_hist = torch.stack(hist) if hist else torch.zeros(0, B, dtype=torch.float64)
    return q, t, dt_hist


def rollout(q0, p: FaceNetParams, dt, T: int, g=9.81, round_bf16=True):
    """States after steps 1..T at the fixed step dt (list of T tensors)."""
    q = q0
    out = []
    for _ in range(T):
        q = step(q, p, dt, g, round_bf16)
        out.append(q)
    return out


def loss_and_grads(q0, targets, p: FaceNetParams, dt, scale, g=9.81, round_bf16=True, want_dq0=False):
    """Rollout loss (Eq. 2.28, the same per-variable scaling as the fourth
    approach) of a T-step rollout and its gradient with respect to the flat
    parameter vector (and, with want_dq0, the initial state), by reverse-mode
    differentiation of this FP64 forward.  Returns (loss, dparams) or
    (loss, dparams, dq0)."""
    from .stencil_net import rollout_loss
    flat = p.flat().detach().clone().requires_grad_(True)
    pp = FaceNetParams.from_flat(flat, p.mean, p.std)
    q0 = torch.as_tensor(q0, dtype=torch.float64).clone().requires_grad_(want_dq0)
    preds = rollout(q0, pp, dt, len(targets), g, round_bf16)
    loss = rollout_loss(preds, targets, scale)
    loss.backward()
    out = (float(loss.detach()), flat.grad.detach().clone())
    return out + (q0.grad.detach().clone(),) if want_dq0 else out


def init_params(seed: int, mean, std, scale: float = 1.0) -> FaceNetParams:
    """He-style random weights (bfloat16 values) and small FP32 biases."""
    gen = torch.Generator().manual_seed(seed)
    W, b = [], []
    for co, ci in LAYER_SHAPES:
        std_w = scale * (2.0 / (ci * 9)) ** 0.5
        w = torch.randn(co, ci, 3, 3, generator=gen, dtype=torch.float64) * std_w
        bb = torch.randn(co, generator=gen, dtype=torch.float64) * 0.01
        W.append(w.to(torch.bfloat16).to(torch.float64))
        b.append(f32(bb))
    return FaceNetParams(W, b, f32(torch.as_tensor(mean, dtype=torch.float64)),
                         f32(torch.as_tensor(std, dtype=torch.float64)))
