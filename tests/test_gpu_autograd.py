"""The learned rollout as a torch.autograd.Function (fv.TapeRollout over
fv_tape_forward / fv_tape_backward) against central finite differences of
the GPU forward itself, along random directions.

Loss: L = sum_t <w_t, q_t> over the T = 2 step snapshots with fixed random
weights w (FP64 accumulation), so that dL/dsnaps = w is the cotangent the
Function's backward receives.  Directions and their step sizes:
  * FP32 directions, through a network whose last-layer weights are zero
    (its stencils are the constants its last-layer biases set, so no
    derivative passes through a BF16 layer): the last layer's biases (added
    in FP32 after the tensor cores; coefficients, learned faces, HLL and the
    RK combine are FP32) and the initial state.  Steps: at most 0.1 on a
    bias, 1e-3 on a depth; tolerance 1e-3 relative (L2 over the directions).
  * BF16 directions: all parameters (multiplicative, 3 % per weight) and the
    initial state through a full random network.  Weights and activations are
    rounded to BF16 on the way to the tensor cores, so the forward is a
    staircase at the 2^-9 relative scale and the step must be much larger than
    that; the backward differentiates the rounding as the identity.
    Tolerance 5e-2 relative (L2 over the directions).
"""
import numpy as np
import pytest
import torch

from helpers import f32
from oracle import stencil_net as osn
from paper_2602_08670_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MEAN = [1.05, 0.0, 0.0]
STD = [0.05, 0.02, 0.02]
N, B, T, DT = 64, 2, 2, 1e-3
TOL_FP32 = 1e-3
TOL_BF16 = 5e-2


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv as binding
    return binding


def _params(seed, zero_w4=False):
    p = osn.init_params(seed, MEAN, STD, zero_last=False, scale=0.5)
    p.W[3] = (p.W[3] * 0.1).to(torch.bfloat16).to(torch.float64)
    g = torch.Generator().manual_seed(seed + 100)
    p.b[3] = 0.05 * torch.randn(p.b[3].shape, generator=g, dtype=torch.float64)
    if zero_w4:
        p.W[3] = torch.zeros_like(p.W[3])
    return torch.tensor(p.flat().numpy().astype(np.float32)).cuda()


def _state(seed):
    q = W.swe_random_bumps(N, seed, B)
    q[:, 1:] = 0.02 * np.sin(np.arange(N) * 2 * np.pi / N)[None, None, None, :]
    return f32(W.as_f32_exact(q)).cuda()


def _setup(fv, params):
    net = fv.stencil_net_create(params.cpu().numpy(), MEAN, STD)
    tape = fv.fv_tape_create(net, B, N, N, T, DT)
    g = torch.Generator(device="cuda").manual_seed(7)
    w = torch.randn((T, B, 3, N, N), generator=g, device="cuda", dtype=torch.float64)
    return tape, w


def _loss(fv, tape, w, params, q0):
    return float((fv.tape_rollout(tape, params, q0).double() * w).sum())


def _grads(fv, tape, w, params, q0):
    p = params.clone().requires_grad_(True)
    q = q0.clone().requires_grad_(True)
    snaps = fv.tape_rollout(tape, p, q)
    (snaps.double() * w).sum().backward()
    return p.grad.clone(), q.grad.clone()


def _fd(fv, tape, w, params, q0, dp, dq, eps):
    lp = _loss(fv, tape, w, params + eps * dp, q0 + eps * dq)
    lm = _loss(fv, tape, w, params - eps * dp, q0 - eps * dq)
    return (lp - lm) / (2 * eps)


def _check(fv, tape, w, params, q0, dirs, tol):
    """Relative L2 over the directions of (finite difference - autograd) of
    the directional derivatives.  `dirs` holds (dparams, dq0, eps) or
    ("grad", scale, eps): a direction along the autograd gradient itself,
    scaled per component by U[0.5, 1.5] (its derivative cannot vanish)."""
    gp, gq = _grads(fv, tape, w, params, q0)
    gen = torch.Generator(device="cuda").manual_seed(99)
    ad, fd = [], []
    for dp, dq, eps in dirs:
        if isinstance(dp, str):
            dp = gp * (0.5 + torch.rand(gp.shape, generator=gen, device="cuda")) * dq
            dq = torch.zeros_like(q0)
            # largest parameter change: 1 % of the largest parameter
            eps = 1e-2 * float(params.abs().max()) / float(dp.abs().max())
        ad.append(float((gp.double() * dp.double()).sum() + (gq.double() * dq.double()).sum()))
        fd.append(_fd(fv, tape, w, params, q0, dp, dq, eps))
    ad, fd = np.array(ad), np.array(fd)
    err = float(np.linalg.norm(fd - ad) / np.linalg.norm(fd))
    assert err <= tol, (err, list(zip(fd.tolist(), ad.tolist())))


def test_autograd_matches_finite_differences_fp32_directions(fv):
    # zero last-layer weights: the stencils are the constants set by the
    # last layer's biases, so no derivative passes through the BF16 layers
    # (with random last-layer weights a bias change of stage 1 reaches the
    # next stage's CNN input, whose cotangents are BF16)
    gen = torch.Generator(device="cuda").manual_seed(11)
    params = _params(6, zero_w4=True)
    tape, w = _setup(fv, params)
    q0 = _state(21)
    nb4 = 36
    dirs = []
    for _ in range(3):
        dp = torch.zeros_like(params)
        dp[-nb4:] = torch.randn(nb4, generator=gen, device="cuda")
        dirs.append((dp, torch.zeros_like(q0), 1e-1 / float(dp.abs().max())))
    for _ in range(3):
        dq = torch.randn(q0.shape, generator=gen, device="cuda")
        dq[:, 0] *= 0.05
        dq[:, 1:] *= 0.02
        dirs.append((torch.zeros_like(params), dq, 1e-3 / float(dq[:, 0].abs().max())))
    _check(fv, tape, w, params, q0, dirs, TOL_FP32)


def test_autograd_matches_finite_differences_bf16_directions(fv):
    gen = torch.Generator(device="cuda").manual_seed(12)
    params = _params(8)
    tape, w = _setup(fv, params)
    q0 = _state(22)
    dirs = []
    for _ in range(3):
        dp = params * torch.randn(params.shape, generator=gen, device="cuda")
        dirs.append((dp, torch.zeros_like(q0), 3e-2))
    # along the gradient: 3 % of the largest parameter change per unit
    dirs.append(("grad", 1.0, None))
    for _ in range(2):
        dq = torch.randn(q0.shape, generator=gen, device="cuda")
        dq[:, 0] *= 0.05
        dq[:, 1:] *= 0.02
        dirs.append((torch.zeros_like(params), dq, 0.3))
    _check(fv, tape, w, params, q0, dirs, TOL_BF16)


def test_autograd_backward_needs_its_own_forward(fv):
    params = _params(6)
    tape, w = _setup(fv, params)
    q0 = _state(21)
    p = params.clone().requires_grad_(True)
    snaps = fv.tape_rollout(tape, p, q0)
    fv.tape_rollout(tape, params, q0)          # the tape now holds another window
    with pytest.raises(RuntimeError, match="recorded another rollout"):
        (snaps.double() * w).sum().backward()
