"""FP64 oracle of the learned-stencil variant (test infrastructure only).

Section 2.5.3, the fourth approach (reconstruction with CNN-generated linear
coefficients; results in Section 5.4): a CNN maps the cell-average
state to constrained coefficients; the face values are those coefficients
applied to the neighbouring cell values; the same flux, divergence and
SSP-RK2 as the plain scheme follow.  Training minimises the rollout loss of
Eq. 2.28 with the solver inside the loss (model-consistent training).

Readings where the paper is silent (each one is listed with its reason in the
design notes):
  * Network: x = (q - mean) / scale per channel (the training set's mean and
    largest absolute deviation); four 3x3 convolutions with
    circular padding, 3 -> 32 -> 32 -> 32 -> 36 channels, ReLU after the
    first three, the last one linear.
  * 36 outputs per cell = 2 directions x 3 variables x 2 sides x 3 taps.  Cell
    i owns face i+1/2 in x and face j+1/2 in y.  Side L uses cells
    {i-1, i, i+1}, side R uses {i, i+1, i+2} (three stencils per face, Section 6.2).
  * Normalisation: w = e_centre + r - mean(r) over the three taps, so the
    weights sum to one and a zero raw output gives the first-order
    (piecewise constant) scheme, the first-order starting point that the
    initialisation of Section 2.5.3 is meant to guarantee.
  * Positivity: where either reconstructed depth at a face is below h_min,
    that face uses the MUSCL-minmod states instead (the plain step is the
    fallback).
  * The CNN runs at every Runge-Kutta stage (the reconstruction is part of
    L(q)).
  * Loss: sum over steps t = 1..T of the per-variable MSE divided by that
    variable's squared scale, summed over variables.

Precision mirror: with ``round_bf16=True`` the network input and every hidden
activation are rounded to bfloat16 and the weights are bfloat16 values, as on
the GPU; sums stay FP64.  Derivatives treat the rounding as the identity.
Finite-difference checks use ``round_bf16=False``.
"""
from __future__ import annotations

import dataclasses

import torch
import torch.nn.functional as F

from . import fv

C_SWE = 3
HIDDEN = 32
N_OUT = 36           # 2 directions x 3 variables x 2 sides x 3 taps
LAYER_SHAPES = [(HIDDEN, C_SWE), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (N_OUT, HIDDEN)]


def out_channel(direction: int, var: int, side: int, tap: int) -> int:
    """Index of one coefficient among the 36 outputs of a cell."""
    return ((direction * C_SWE + var) * 2 + side) * 3 + tap


def bf16(x: torch.Tensor) -> torch.Tensor:
    """Round to bfloat16 (nearest-even) and back, keeping the graph."""
    return x + (x.detach().to(torch.float32).to(torch.bfloat16).to(torch.float64) - x.detach())


def f32(x: torch.Tensor) -> torch.Tensor:
    return x.detach().to(torch.float32).to(torch.float64)


@dataclasses.dataclass
class NetParams:
    W: list            # 4 tensors [Cout][Cin][3][3]
    b: list            # 4 tensors [Cout]
    mean: torch.Tensor  # [3]
    std: torch.Tensor   # [3]

    def params(self):
        return self.W + self.b

    @staticmethod
    def from_flat(flat: torch.Tensor, mean, std) -> "NetParams":
        """Unpack the flat parameter vector: W1, b1, W2, b2, W3, b3, W4, b4."""
        W, b, off = [], [], 0
        for co, ci in LAYER_SHAPES:
            n = co * ci * 9
            W.append(flat[off:off + n].reshape(co, ci, 3, 3).clone())
            off += n
            b.append(flat[off:off + co].clone())
            off += co
        return NetParams(W, b, torch.as_tensor(mean, dtype=torch.float64),
                         torch.as_tensor(std, dtype=torch.float64))

    def flat(self) -> torch.Tensor:
        parts = []
        for W, b in zip(self.W, self.b):
            parts += [W.reshape(-1), b.reshape(-1)]
        return torch.cat(parts)


def n_params() -> int:
    return sum(co * ci * 9 + co for co, ci in LAYER_SHAPES)


def conv3x3_periodic(x: torch.Tensor, W: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """y[co] = b[co] + sum_{ci, dy, dx} W[co, ci, dy+1, dx+1] x[ci](j+dy, i+dx),
    neighbours taken periodically (cross-correlation, as in every CNN library)."""
    return F.conv2d(F.pad(x, (1, 1, 1, 1), mode="circular"), W, b)


def conv3x3_periodic_loops(x: torch.Tensor, W: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """The same convolution written out as loops (for pinning on tiny inputs)."""
    B, Ci, ny, nx = x.shape
    Co = W.shape[0]
    y = torch.zeros(B, Co, ny, nx, dtype=x.dtype)
    for bb in range(B):
        for co in range(Co):
            for j in range(ny):
                for i in range(nx):
                    s = float(b[co])
                    for ci in range(Ci):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                s += float(W[co, ci, dy + 1, dx + 1]) * \
                                    float(x[bb, ci, (j + dy) % ny, (i + dx) % nx])
                    y[bb, co, j, i] = s
    return y


def net_raw(q: torch.Tensor, p: NetParams, round_bf16: bool = True) -> torch.Tensor:
    """Raw network output r[B][36][ny][nx] for the state q (SWE)."""
    x = (q - p.mean.view(1, -1, 1, 1)) / p.std.view(1, -1, 1, 1)
    if round_bf16:
        x = bf16(x)
    for layer in range(4):
        x = conv3x3_periodic(x, p.W[layer], p.b[layer])
        if layer < 3:
            x = torch.relu(x)
            if round_bf16:
                x = bf16(x)
    return x


def normalise(raw: torch.Tensor) -> torch.Tensor:
    """w = e_centre + r - mean_taps(r) for every (direction, variable, side):
    the three weights of each stencil sum to one."""
    B, _, ny, nx = raw.shape
    r = raw.reshape(B, 2, C_SWE, 2, 3, ny, nx)
    e = torch.zeros(3, dtype=raw.dtype)
    e[1] = 1.0
    w = e.view(1, 1, 1, 1, 3, 1, 1) + r - r.mean(dim=4, keepdim=True)
    return w.reshape(B, N_OUT, ny, nx)


def learned_faces(Q: torch.Tensor, w: torch.Tensor, direction: int, dim: int):
    """Face states at i+1/2 (index i) along ``dim`` from the owner cell's
    weights: Q^L = sum_k wL_k Q_{i-1+k},  Q^R = sum_k wR_k Q_{i+k}."""
    B, C, ny, nx = Q.shape
    wd = w.reshape(B, 2, C, 2, 3, ny, nx)[:, direction]   # [B][var][side][tap]
    Qm = torch.roll(Q, 1, dims=dim)
    Qp = torch.roll(Q, -1, dims=dim)
    Qpp = torch.roll(Q, -2, dims=dim)
    QL = wd[:, :, 0, 0] * Qm + wd[:, :, 0, 1] * Q + wd[:, :, 0, 2] * Qp
    QR = wd[:, :, 1, 0] * Q + wd[:, :, 1, 1] * Qp + wd[:, :, 1, 2] * Qpp
    return QL, QR


def faces_with_fallback(Q, w, direction, dim, delta, h_min):
    """Learned faces, replaced by MUSCL-minmod faces wherever a learned face
    depth falls below ``h_min`` (per member, shape [B])."""
    QL, QR = learned_faces(Q, w, direction, dim)
    hm = torch.as_tensor(h_min, dtype=Q.dtype).reshape(-1, 1, 1)
    bad = ((QL[:, 0] < hm) | (QR[:, 0] < hm)).unsqueeze(1)
    mL, mR = fv.muscl_minmod(Q, dim, delta)
    return torch.where(bad, mL, QL), torch.where(bad, mR, QR)


def learned_rhs(q, p: NetParams, dx, dy, h_min, g=9.81, round_bf16=True, weights=None):
    """L(q) with CNN coefficients (or the given ``weights``) in place of
    MUSCL-minmod; flux and divergence as in the plain scheme."""
    w = normalise(net_raw(q, p, round_bf16)) if weights is None else weights
    QLx, QRx = faces_with_fallback(q, w, 0, -1, dx, h_min)
    Fx = fv.face_flux(QLx, QRx, *fv.X_FACE, fv.SWE, g, 1.4)
    QLy, QRy = faces_with_fallback(q, w, 1, -2, dy, h_min)
    Gy = fv.face_flux(QLy, QRy, *fv.Y_FACE, fv.SWE, g, 1.4)
    return fv.divergence_update(Fx, Gy, dx, dy)


def learned_step(q, p: NetParams, dt, h_min, g=9.81, round_bf16=True):
    dx, dy = fv.grid_spacing(q)
    return fv.ssp_rk2(q, dt, lambda s: learned_rhs(s, p, dx, dy, h_min, g, round_bf16))


def rollout(q0, p: NetParams, dt, T: int, h_min, g=9.81, round_bf16=True):
    """States after steps 1..T (list of T tensors)."""
    q = q0
    out = []
    for _ in range(T):
        q = learned_step(q, p, dt, h_min, g, round_bf16)
        out.append(q)
    return out


def rollout_loss(preds, targets, scale) -> torch.Tensor:
    """Eq. 2.28: sum_t MSE(Q_exact(t), Q_pred(t)), each variable's squared
    error divided by scale[c]^2 before the mean, variables summed."""
    s = torch.as_tensor(scale, dtype=torch.float64).view(1, -1, 1, 1)
    total = torch.zeros((), dtype=torch.float64)
    for qp, qe in zip(preds, targets):
        d = (qp - qe) / s
        total = total + (d * d).mean(dim=(0, 2, 3)).sum()
    return total


def loss_and_grads(q0, targets, p: NetParams, dt, h_min, scale, g=9.81,
                   round_bf16=True, want_dq0=False):
    """Loss (2.28) of a T-step rollout and its gradient with respect to the
    flat parameter vector (and optionally q0), by reverse-mode
    differentiation of this FP64 forward."""
    flat = p.flat().clone().requires_grad_(True)
    # views into `flat`, so that gradients flow to it
    W, b, off = [], [], 0
    for co, ci in LAYER_SHAPES:
        n = co * ci * 9
        W.append(flat[off:off + n].reshape(co, ci, 3, 3))
        off += n
        b.append(flat[off:off + co])
        off += co
    pp = NetParams(W, b, p.mean, p.std)
    q0 = torch.as_tensor(q0, dtype=torch.float64).clone().requires_grad_(want_dq0)
    preds = rollout(q0, pp, dt, len(targets), h_min, g, round_bf16)
    loss = rollout_loss(preds, targets, scale)
    loss.backward()
    return float(loss.detach()), flat.grad.detach().clone(), (q0.grad.detach().clone() if want_dq0 else None)


def init_params(seed: int, mean, std, zero_last: bool = True, scale: float = 1.0) -> NetParams:
    """He-style random init; a zero last layer makes the network start as the
    first-order scheme.  Weights are rounded to bfloat16, biases to FP32."""
    g = torch.Generator().manual_seed(seed)
    W, b = [], []
    for layer, (co, ci) in enumerate(LAYER_SHAPES):
        std_w = scale * (2.0 / (ci * 9)) ** 0.5
        w = torch.randn(co, ci, 3, 3, generator=g, dtype=torch.float64) * std_w
        bb = torch.randn(co, generator=g, dtype=torch.float64) * 0.01
        if layer == 3 and zero_last:
            w.zero_()
            bb.zero_()
        W.append(w.to(torch.bfloat16).to(torch.float64))
        b.append(f32(bb))
    return NetParams(W, b, f32(torch.as_tensor(mean, dtype=torch.float64)),
                     f32(torch.as_tensor(std, dtype=torch.float64)))
