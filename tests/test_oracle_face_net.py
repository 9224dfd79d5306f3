"""Pins of the face-state CNN oracle (``oracle.face_net``, Section 2.5.3's
third approach): GeLU and Softplus against tabulated values and identities,
the side-state layout and tap orientation through a hand-built network, the
flux pairing against the plain MUSCL-minmod and first-order schemes, depth
positivity, translation equivariance, conservation, and reverse-mode
gradients against central finite differences.  CPU only."""
import math

import numpy as np
import pytest
import torch

from oracle import face_net as fn
from oracle import fv
from paper_2602_08670_gb300 import workloads as W

MEAN = [1.05, 0.0, 0.0]
STD = [0.05, 0.02, 0.02]


def test_gelu_tabulated():
    """x Phi(x) with the tabulated normal distribution Phi(1) = 0.841344746,
    Phi(2) = 0.977249868, Phi(-0.5) = 0.308537539; GeLU(x) - GeLU(-x) = x."""
    x = torch.tensor([1.0, 2.0, -0.5, 0.0], dtype=torch.float64)
    ref = torch.tensor([0.8413447460685429, 2 * 0.9772498680518208, -0.5 * 0.3085375387259869, 0.0],
                       dtype=torch.float64)
    assert torch.allclose(fn.gelu(x), ref, rtol=0, atol=1e-15)
    y = torch.linspace(-6, 6, 101, dtype=torch.float64)
    assert torch.allclose(fn.gelu(y) - fn.gelu(-y), y, rtol=0, atol=1e-14)


def test_softplus_identities():
    x = torch.linspace(-40, 40, 161, dtype=torch.float64)
    assert abs(float(fn.softplus(torch.zeros(1, dtype=torch.float64))) - math.log(2.0)) < 1e-16
    assert torch.allclose(fn.softplus(x) - fn.softplus(-x), x, rtol=0, atol=1e-13)
    big = torch.tensor([800.0, -800.0, -30.0], dtype=torch.float64)
    s = fn.softplus(big)
    assert float(s[0]) == 800.0 and float(s[1]) >= 0.0
    assert abs(float(s[2]) - math.exp(-30.0)) < 1e-25


def muscl_sides(q, dx, dy):
    """Side states of the MUSCL-minmod reconstruction (Eq. 2.18):
    Q_i -/+ s_i d / 2 on the west/east (south/north) sides."""
    sx = fv.minmod((q - torch.roll(q, 1, -1)) / dx, (torch.roll(q, -1, -1) - q) / dx)
    sy = fv.minmod((q - torch.roll(q, 1, -2)) / dy, (torch.roll(q, -1, -2) - q) / dy)
    return torch.stack([q - sx * dx / 2, q + sx * dx / 2, q - sy * dy / 2, q + sy * dy / 2], dim=1)


def random_swe(B, ny, nx, seed):
    return torch.tensor(W.random_smooth_swe(nx, seed, members=B)[:, :, :ny, :nx])


def test_face_rhs_with_muscl_sides_is_the_plain_scheme():
    """Fed the MUSCL-minmod side states, the face-state right-hand side is the
    plain scheme's, bit for bit: each face pairs the east (north) state of
    the cell before it with the west (south) state of the cell after it.  A
    swapped pairing or a roll the wrong way breaks this."""
    q = random_swe(2, 12, 16, 3)
    q[:, 1:] += 0.05 * torch.randn(2, 2, 12, 16, generator=torch.Generator().manual_seed(1), dtype=torch.float64)
    dx, dy = fv.grid_spacing(q)
    a = fn.face_rhs(q, muscl_sides(q, dx, dy).reshape(2, 4, 3, 12, 16), dx, dy)
    b = fv.rhs(q, fv.SWE, dx, dy)
    assert torch.equal(a, b)


def test_face_rhs_with_cell_values_is_first_order():
    q = random_swe(1, 8, 10, 4)
    dx, dy = fv.grid_spacing(q)
    sides = q.unsqueeze(1).expand(1, 4, 3, 8, 10)
    a = fn.face_rhs(q, sides, dx, dy)
    b = fv.rhs(q, fv.SWE, dx, dy, recon=lambda Q, dim, d: fv.first_order_faces(Q, dim))
    assert torch.equal(a, b)


SHIFT = 40.0   # GeLU(y) = y to FP64 precision for y >= 37


def passthrough_params(side_taps):
    """A hand-built network: the hidden layers carry the three normalised
    inputs shifted by +40 (where GeLU is the identity), and output channel
    (side, var) reads input var at the tap side_taps[side] = (dy, dx)."""
    p = fn.FaceNetParams.from_flat(torch.zeros(fn.n_params(), dtype=torch.float64), MEAN, STD)
    W = [w.clone() for w in p.W]
    b = [x.clone() for x in p.b]
    for v in range(3):
        W[0][v, v, 1, 1] = 1.0
        b[0][v] = SHIFT
        for layer in (1, 2):
            W[layer][v, v, 1, 1] = 1.0
    for s, (dy, dx) in enumerate(side_taps):
        for v in range(3):
            W[3][fn.out_channel(s, v), v, dy + 1, dx + 1] = 1.0
            b[3][fn.out_channel(s, v)] = -SHIFT
    return fn.FaceNetParams(W, b, p.mean, p.std)


def test_side_layout_and_tap_orientation():
    """Output channel 3 s + v is side s of variable v; the network's tap
    (dy, dx) reads the cell (j + dy, i + dx); momenta come back
    de-normalised (mean + std r) and depths through Softplus."""
    q = random_swe(1, 6, 7, 5)
    taps = [(0, -1), (0, 1), (-1, 0), (1, 0)]     # each side reads the neighbour behind it
    p = passthrough_params(taps)
    sides = fn.side_states(fn.net_raw(q, p, round_bf16=False), p).reshape(1, 4, 3, 6, 7)
    mean = torch.tensor(MEAN, dtype=torch.float64).view(1, 3, 1, 1)
    std = torch.tensor(STD, dtype=torch.float64).view(1, 3, 1, 1)
    for s, (dy, dx) in enumerate(taps):
        nb = torch.roll(q, (-dy, -dx), (-2, -1))
        assert torch.allclose(sides[:, s, 1:], nb[:, 1:], rtol=0, atol=1e-13), s
        xh = (nb[:, 0] - mean[:, 0]) / std[:, 0]
        assert torch.allclose(sides[:, s, 0], torch.log1p(torch.exp(xh)), rtol=1e-13, atol=0), s


def test_depths_are_positive_for_any_network():
    """Softplus keeps every reconstructed depth positive, whatever the
    weights (here biased to drive the raw depth outputs far negative), as
    long as e^r does not underflow (r > -745 in FP64, about -87 in FP32)."""
    q = random_swe(2, 8, 8, 6)
    p = fn.init_params(3, MEAN, STD, scale=2.0)
    p.b[3][0::3] -= 30.0
    sides = fn.side_states(fn.net_raw(q, p), p)
    assert bool((sides[:, :, 0] > 0).all())
    assert float(sides[:, :, 0].min()) < 1e-9


def test_translation_equivariance():
    q = random_swe(1, 8, 12, 7)
    p = fn.init_params(4, MEAN, STD)
    r = fn.net_raw(q, p, round_bf16=False)
    r2 = fn.net_raw(torch.roll(q, (3, -5), (-2, -1)), p, round_bf16=False)
    assert torch.allclose(torch.roll(r, (3, -5), (-2, -1)), r2, rtol=0, atol=1e-12)


def test_step_conserves_mass_and_keeps_a_lake_at_rest():
    """Mass: the update is conservative for any side states.  Lake at rest:
    a network that outputs the resting state on every side (zero weights,
    biases softplus^-1(h0) and zero momenta) leaves it unchanged bitwise."""
    q = random_swe(2, 8, 8, 8)
    p = fn.init_params(5, MEAN, STD)
    q1 = fn.step(q, p, torch.tensor([2e-3, 1e-3], dtype=torch.float64).view(2, 1, 1, 1))
    assert torch.allclose(q1[:, 0].sum(dim=(-1, -2)), q[:, 0].sum(dim=(-1, -2)), rtol=1e-14, atol=0)
    h0 = 1.25
    rest = torch.zeros(1, 3, 8, 8, dtype=torch.float64)
    rest[:, 0] = h0
    z = fn.FaceNetParams.from_flat(torch.zeros(fn.n_params(), dtype=torch.float64), [0, 0, 0], [1, 1, 1])
    b3 = z.b[3].clone()
    b3[0::3] = math.log(math.expm1(h0))
    z = fn.FaceNetParams(z.W, z.b[:3] + [b3], z.mean, z.std)
    out = fn.step(rest, z, 1e-3, round_bf16=False)
    assert torch.allclose(out, rest, rtol=0, atol=1e-15)


def test_gradients_match_finite_differences():
    q0 = random_swe(1, 8, 8, 9)
    p = fn.init_params(6, MEAN, STD, scale=0.5)
    targets = [q0 + 0.001 * k for k in (1, 2)]
    scale = [0.05, 0.02, 0.02]
    dt = 1e-3
    loss, grad = fn.loss_and_grads(q0, targets, p, dt, scale, round_bf16=False)
    flat = p.flat().detach()
    rng = np.random.default_rng(0)
    idx = list(rng.choice(flat.numel(), 6, replace=False)) + [flat.numel() - 1, flat.numel() - 13]
    for i in idx:
        eps = 1e-6
        f1 = flat.clone()
        f1[i] += eps
        f2 = flat.clone()
        f2[i] -= eps
        l1, _ = fn.loss_and_grads(q0, targets, fn.FaceNetParams.from_flat(f1, MEAN, STD), dt, scale, round_bf16=False)
        l2, _ = fn.loss_and_grads(q0, targets, fn.FaceNetParams.from_flat(f2, MEAN, STD), dt, scale, round_bf16=False)
        fd = (l1 - l2) / (2 * eps)
        assert abs(fd - float(grad[i])) <= 1e-6 * max(1.0, abs(fd)), (i, fd, float(grad[i]))


def test_run_replay_equals_adaptive():
    q0 = random_swe(1, 8, 8, 10)
    p = fn.init_params(7, MEAN, STD, scale=0.3)
    qa, ta, dts = fn.run(q0, p, 4)
    qr, tr, _ = fn.run(q0, p, 4, dt_mode=fv.DT_REPLAY, dts=dts[:, 0])
    assert torch.equal(qa, qr) and torch.equal(ta, tr)
