"""Parity of the learned-stencil path with the FP64 oracle: the tcgen05 CNN
forward (raw outputs and normalised coefficients), and the learned SSP-RK2
step with the special weights that reduce it to textbook schemes, with a
random network, and with the positivity fallback.  Calls go through the C ABI."""
import numpy as np
import pytest
import torch

from helpers import f32, rel_errors
from oracle import fv as ofv
from oracle import stencil_net as osn
from paper_2602_08670_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MEAN = [1.05, 0.0, 0.0]
STD = [0.05, 0.02, 0.02]
# FP32 roundoff after <= 20 steps (same yardstick as the plain step): depth
# to 1e-5 / 1e-4 (relative L2 / Linf), the small momenta to 1e-4 / 1e-4.
TOLS = [(1e-5, 1e-4), (1e-4, 1e-4), (1e-4, 1e-4)]


def check(err, tols=TOLS):
    for c, ((e2, ei), (l2, li)) in enumerate(zip(err, tols)):
        assert e2 <= l2 and ei <= li, (c, e2, ei, err)


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv as binding
    return binding


def rand_params(seed, last_scale=1.0, scale=0.5):
    p = osn.init_params(seed, MEAN, STD, zero_last=False, scale=scale)
    p.W[3] = (p.W[3] * last_scale).to(torch.bfloat16).to(torch.float64)
    return p


def gpu_net(fv, p):
    return fv.stencil_net_create(p.flat().numpy().astype(np.float32), MEAN, STD)


def swe_state(n, seed, members=2):
    q = W.swe_random_bumps(n, seed, members)
    q[:, 1:] = 0.02 * np.sin(np.arange(n) * 2 * np.pi / n)[None, None, None, :]
    return W.as_f32_exact(q)


@pytest.mark.parametrize("ny,nx", [(64, 64), (16, 128), (32, 256), (16, 8)])
def test_cnn_raw_matches_oracle(fv, ny, nx):
    p = rand_params(1)
    net = gpu_net(fv, p)
    q0 = W.as_f32_exact(W.random_smooth_swe(max(nx, ny), seed=3, members=2, vel=0.2)[:, :, :ny, :nx])
    raw = fv.stencil_net_forward(net, f32(q0).cuda(), raw=True).double().cpu()
    ref = osn.net_raw(torch.tensor(q0), p, round_bf16=True).detach()
    scale = float(ref.abs().max())
    err = (raw - ref).abs()
    # BF16 activations on both sides; FP32 (GPU) vs FP64 (oracle) sums can flip
    # a BF16 rounding now and then, each worth 2^-9 of one of 288 terms
    assert float(err.max()) <= 1e-2 * scale, (float(err.max()), scale)
    assert float(err.mean()) <= 1e-3 * scale, (float(err.mean()), scale)


def test_cnn_coefficients_normalised(fv):
    p = rand_params(2)
    net = gpu_net(fv, p)
    q0 = swe_state(64, 5)
    w = fv.stencil_net_forward(net, f32(q0).cuda()).double().cpu()
    ref = osn.normalise(osn.net_raw(torch.tensor(q0), p, round_bf16=True)).detach()
    assert float((w - ref).abs().max()) <= 1e-2 * float(ref.abs().max())
    sums = w.reshape(2, 12, 3, 64, 64).sum(dim=2)
    assert float((sums - 1).abs().max()) < 1e-6


def test_zero_network_is_first_order(fv):
    net = fv.stencil_net_create(None, MEAN, STD)
    q0 = swe_state(64, 7)
    w = fv.stencil_net_forward(net, f32(q0).cuda()).cpu()
    e = torch.zeros(36)
    e[1::3] = 1.0
    assert torch.equal(w, e.view(1, 36, 1, 1).expand_as(w))
    s = fv.swe_init(f32(q0).cuda(), dt_mode="fixed", dt_fixed=2e-4)
    fv.fv_rollout(s, 20, net=net)
    q = fv.fv_get_state(s).double().cpu()
    first = lambda Q, d, delta: ofv.first_order_faces(Q, d)
    qr, _, _, _ = ofv.run(torch.tensor(q0), ofv.SWE, 20, dt_mode=ofv.DT_FIXED, dt_fixed=2e-4, recon=first)
    check(rel_errors(q, qr))


def fromm_params():
    p = osn.init_params(0, MEAN, STD, zero_last=True)
    b4 = torch.zeros(36, dtype=torch.float64)
    for d in range(2):
        for v in range(3):
            b4[osn.out_channel(d, v, 0, 0)] = -0.25
            b4[osn.out_channel(d, v, 0, 2)] = 0.25
            b4[osn.out_channel(d, v, 1, 0)] = 0.25
            b4[osn.out_channel(d, v, 1, 2)] = -0.25
    p.b[3] = b4
    return p


def test_fromm_weights_give_unlimited_linear_scheme(fv):
    p = fromm_params()
    net = gpu_net(fv, p)
    q0 = swe_state(64, 9)
    s = fv.swe_init(f32(q0).cuda(), dt_mode="fixed", dt_fixed=2e-4)
    fv.fv_rollout(s, 20, net=net)
    q = fv.fv_get_state(s).double().cpu()

    def fromm(Q, dim, delta):
        Qm, Qp, Qpp = (torch.roll(Q, k, dim) for k in (1, -1, -2))
        return Q + (Qp - Qm) / 4, Qp - (Qpp - Q) / 4
    qr, _, _, _ = ofv.run(torch.tensor(q0), ofv.SWE, 20, dt_mode=ofv.DT_FIXED, dt_fixed=2e-4, recon=fromm)
    check(rel_errors(q, qr))


def test_learned_step_random_network_matches_oracle(fv):
    p = rand_params(4, last_scale=0.1)
    net = gpu_net(fv, p)
    q0 = swe_state(64, 11)
    s = fv.swe_init(f32(q0).cuda(), dt_mode="fixed", dt_fixed=2e-4)
    fv.fv_rollout(s, 10, net=net)
    q = fv.fv_get_state(s).double().cpu()
    hmin = torch.tensor(1e-3 * q0[:, 0].mean(axis=(1, 2)))
    qr = torch.tensor(q0)
    for _ in range(10):
        qr = osn.learned_step(qr, p, 2e-4, hmin, round_bf16=True).detach()
    for c, (e2, ei) in enumerate(rel_errors(q, qr)):
        assert e2 < 1e-4 and ei < 1e-3, (c, e2, ei)


def test_positivity_fallback_matches_oracle(fv):
    p = fromm_params()
    p.b[3] = p.b[3] * 24.0          # strongly extrapolating stencils
    net = gpu_net(fv, p)
    q0 = swe_state(64, 13)
    s = fv.swe_init(f32(q0).cuda(), dt_mode="fixed", dt_fixed=1e-4)
    fv.fv_set_learned_hmin(s, 0.97)   # h_min just below the minimum depth: many faces fall back
    fv.fv_rollout(s, 5, net=net)
    q = fv.fv_get_state(s).double().cpu()
    hmin = torch.tensor(0.97 * q0[:, 0].mean(axis=(1, 2)))
    qr = torch.tensor(q0)
    for _ in range(5):
        qr = osn.learned_step(qr, p, 1e-4, hmin, round_bf16=True).detach()
    for c, (e2, ei) in enumerate(rel_errors(q, qr)):
        assert e2 < 1e-4 and ei < 1e-3, (c, e2, ei)


def test_unsupported_grid_rejected(fv):
    net = fv.stencil_net_create(None, MEAN, STD)
    with pytest.raises(fv.FvError) as ei:
        fv.stencil_net_forward(net, torch.ones(1, 3, 100, 100, device="cuda"))
    assert ei.value.code == fv.FV_EINVAL
