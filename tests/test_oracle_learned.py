"""Pins of the learned-stencil oracle: the convolution against its loop
definition, the sum-to-one normalisation, the special weights that reduce the
learned reconstruction to textbook schemes (first order; unlimited Fromm),
the positivity fallback, the rollout loss (Eq. 2.28) and reverse-mode
gradients against central finite differences.  CPU only."""
import numpy as np
import pytest
import torch

from oracle import fv
from oracle import stencil_net as sn
from paper_2602_08670_gb300 import workloads as W

MEAN = [1.05, 0.0, 0.0]
STD = [0.05, 0.02, 0.02]


def test_conv_matches_loop_definition():
    g = torch.Generator().manual_seed(0)
    x = torch.randn(2, 3, 4, 5, generator=g, dtype=torch.float64)
    Wt = torch.randn(2, 3, 3, 3, generator=g, dtype=torch.float64)
    b = torch.randn(2, generator=g, dtype=torch.float64)
    assert torch.allclose(sn.conv3x3_periodic(x, Wt, b), sn.conv3x3_periodic_loops(x, Wt, b),
                          rtol=1e-13, atol=1e-13)


def test_conv_tap_orientation():
    # a single tap W[0,0,dy+1,dx+1] = 1 reads x at (j+dy, i+dx)
    x = torch.arange(20, dtype=torch.float64).reshape(1, 1, 4, 5)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            Wt = torch.zeros(1, 1, 3, 3, dtype=torch.float64)
            Wt[0, 0, dy + 1, dx + 1] = 1.0
            y = sn.conv3x3_periodic(x, Wt, torch.zeros(1, dtype=torch.float64))
            assert torch.equal(y, torch.roll(x, (-dy, -dx), (-2, -1)))


def test_normalise_sums_to_one_and_zero_is_first_order():
    g = torch.Generator().manual_seed(1)
    raw = torch.randn(2, 36, 3, 4, generator=g, dtype=torch.float64)
    w = sn.normalise(raw).reshape(2, 2, 3, 2, 3, 3, 4)
    assert torch.allclose(w.sum(dim=4), torch.ones(2, 2, 3, 2, 3, 4, dtype=torch.float64),
                          atol=1e-14)
    w0 = sn.normalise(torch.zeros(1, 36, 2, 2, dtype=torch.float64)).reshape(1, 2, 3, 2, 3, 2, 2)
    assert torch.equal(w0[:, :, :, :, 1], torch.ones(1, 2, 3, 2, 2, 2, dtype=torch.float64))
    assert float(w0[:, :, :, :, [0, 2]].abs().max()) == 0.0


def test_channel_index_layout():
    assert sn.out_channel(0, 0, 0, 0) == 0
    assert sn.out_channel(0, 0, 1, 0) == 3
    assert sn.out_channel(0, 1, 0, 0) == 6
    assert sn.out_channel(1, 0, 0, 0) == 18
    assert sn.out_channel(1, 2, 1, 2) == 35
    assert sn.n_params() == 29796


def _const_weights(B, ny, nx, left, right):
    w = torch.zeros(B, 2, 3, 2, 3, ny, nx, dtype=torch.float64)
    w[:, :, :, 0] = torch.tensor(left, dtype=torch.float64).view(3, 1, 1)
    w[:, :, :, 1] = torch.tensor(right, dtype=torch.float64).view(3, 1, 1)
    return w.reshape(B, 36, ny, nx)


def test_zero_network_is_first_order_scheme_bitwise():
    q = torch.tensor(W.random_smooth_swe(16, seed=2, vel=0.2))
    p = sn.init_params(0, MEAN, STD, zero_last=True)
    dx = dy = 1 / 16
    L_learned = sn.learned_rhs(q, p, dx, dy, h_min=torch.tensor([1e-3]))
    L_first = fv.rhs(q, fv.SWE, dx, dy, recon=lambda Q, d, delta: fv.first_order_faces(Q, d))
    assert torch.equal(L_learned, L_first)


def test_fromm_weights_give_unlimited_linear_reconstruction():
    q = torch.tensor(W.random_smooth_swe(12, seed=3, vel=0.2))
    w = _const_weights(1, 12, 12, [-0.25, 1.0, 0.25], [0.25, 1.0, -0.25])
    for direction, dim in ((0, -1), (1, -2)):
        QL, QR = sn.learned_faces(q, w, direction, dim)
        Qm, Qp, Qpp = (torch.roll(q, s, dim) for s in (1, -1, -2))
        assert torch.allclose(QL, q + (Qp - Qm) / 4, rtol=0, atol=1e-15)
        assert torch.allclose(QR, Qp - (Qpp - q) / 4, rtol=0, atol=1e-15)


def test_learned_reconstruction_exact_on_linear_data():
    n = 12
    x = W.cell_centres(n)
    Q = torch.zeros(1, 3, 1, n, dtype=torch.float64)
    Q[0, 0, 0] = torch.tensor(1.0 + 0.3 * x)
    w = _const_weights(1, 1, n, [-0.25, 1.0, 0.25], [0.25, 1.0, -0.25])
    QL, QR = sn.learned_faces(Q, w, 0, -1)
    face = torch.tensor(1.0 + 0.3 * (np.arange(n) + 1) / n)
    assert torch.allclose(QL[0, 0, 0, 1:n - 2], face[1:n - 2], atol=1e-14)
    assert torch.allclose(QR[0, 0, 0, 1:n - 2], face[1:n - 2], atol=1e-14)


def test_positivity_fallback_uses_minmod_faces():
    q = torch.tensor(W.random_smooth_swe(8, seed=4, vel=0.1))
    # strongly extrapolating weights push some face depths below h_min
    w = _const_weights(1, 8, 8, [-3.0, 1.0, 3.0], [3.0, 1.0, -3.0])
    h_min = torch.tensor([1.0])
    QLl, QRl = sn.learned_faces(q, w, 0, -1)
    bad = (QLl[:, 0] < 1.0) | (QRl[:, 0] < 1.0)
    assert bool(bad.any()) and not bool(bad.all())
    QL, QR = sn.faces_with_fallback(q, w, 0, -1, 1 / 8, h_min)
    mL, mR = fv.muscl_minmod(q, -1, 1 / 8)
    for c in range(3):
        assert torch.equal(QL[:, c][bad], mL[:, c][bad])
        assert torch.equal(QL[:, c][~bad], QLl[:, c][~bad])
        assert torch.equal(QR[:, c][bad], mR[:, c][bad])


def test_rollout_loss_closed_form():
    a = [torch.ones(1, 3, 2, 2, dtype=torch.float64), torch.zeros(1, 3, 2, 2, dtype=torch.float64)]
    b = [torch.zeros(1, 3, 2, 2, dtype=torch.float64)] * 2
    scale = [1.0, 2.0, 4.0]
    # step 1: per-variable MSE 1, 1/4, 1/16; step 2: 0
    assert float(sn.rollout_loss(a, b, scale)) == pytest.approx(1 + 0.25 + 0.0625, rel=1e-15)
    assert float(sn.rollout_loss(b, b, scale)) == 0.0


def _loss_of_flat(flat, q0, targets, dt, h_min, scale):
    p = sn.NetParams.from_flat(flat, MEAN, STD)
    preds = sn.rollout(q0, p, dt, len(targets), h_min, round_bf16=False)
    return float(sn.rollout_loss(preds, targets, scale))


def test_gradients_match_central_differences():
    n, T, dt = 8, 2, 2e-3
    q0 = torch.tensor(W.random_smooth_swe(n, seed=6, members=2, vel=0.2))
    targets = [q0 + 0.01 * torch.randn(q0.shape, generator=torch.Generator().manual_seed(k),
                                       dtype=torch.float64) for k in range(T)]
    p = sn.init_params(3, MEAN, STD, zero_last=False, scale=0.3)
    # shrink the last layer so learned faces stay near first order (no fallback)
    p.W[3] = p.W[3] * 0.05
    h_min = torch.tensor([1e-3, 1e-3])
    scale = [0.05, 0.02, 0.02]
    loss, grad, gq = sn.loss_and_grads(q0, targets, p, dt, h_min, scale, round_bf16=False,
                                       want_dq0=True)
    flat = p.flat()
    g = torch.Generator().manual_seed(9)
    eps = 1e-6
    for _ in range(4):
        d = torch.randn(flat.shape, generator=g, dtype=torch.float64)
        fp = _loss_of_flat(flat + eps * d, q0, targets, dt, h_min, scale)
        fm = _loss_of_flat(flat - eps * d, q0, targets, dt, h_min, scale)
        fd = (fp - fm) / (2 * eps)
        ad = float(grad @ d)
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-12), (fd, ad)
    # gradient with respect to the initial state
    dq = torch.randn(q0.shape, generator=g, dtype=torch.float64)
    pflat = flat
    fp = _loss_of_flat(pflat, q0 + eps * dq, targets, dt, h_min, scale)
    fm = _loss_of_flat(pflat, q0 - eps * dq, targets, dt, h_min, scale)
    fd = (fp - fm) / (2 * eps)
    ad = float((gq * dq).sum())
    assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-12), (fd, ad)


def test_bf16_rounding_mirror():
    x = torch.tensor([1.0, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 3.14159], dtype=torch.float64)
    r = sn.bf16(x)
    assert float(r[0]) == 1.0
    assert float(r[1]) == 1.0                 # tie rounds to even
    assert float(r[2]) == 1.0 + 2 ** -7       # tie rounds to even (up)
    assert float(r[3]) == 3.140625
