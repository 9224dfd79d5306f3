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


@pytest.mark.parametrize("ny,nx", [(64, 64), (16, 128), (32, 256), (16, 8), (5, 128), (6, 64)])
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


def _cos_rel(a, b):
    a = torch.as_tensor(a, dtype=torch.float64).reshape(-1)
    b = torch.as_tensor(b, dtype=torch.float64).reshape(-1)
    cos = float(a @ b / (a.norm() * b.norm()))
    rel = float((a - b).norm() / b.norm())
    return cos, rel


@pytest.mark.parametrize("n,T,B,zero", [(16, 2, 2, True), (16, 2, 2, False), (64, 3, 2, False)])
def test_rollout_gradients_match_oracle(fv, n, T, B, zero):
    """Loss (Eq. 2.28) and its gradient w.r.t. the parameters and the initial
    state through a T-step learned rollout: GPU hand-written backward against
    the oracle's FP64 reverse-mode gradient of the same (BF16-mirrored)
    forward.  zero=True: all-zero network (first-order faces; only b4 has a
    gradient), which isolates the finite-volume adjoint."""
    if zero:
        p = osn.init_params(0, MEAN, STD, zero_last=True)
        for l in range(4):
            p.W[l] = torch.zeros_like(p.W[l])
            p.b[l] = torch.zeros_like(p.b[l])
    else:
        p = rand_params(6, last_scale=0.1)
    dt = 1e-3 if n == 64 else 2e-3
    q0 = swe_state(n, 21, members=B)
    g = torch.Generator().manual_seed(3)
    targets = [torch.tensor(q0) * (1 + 0.01 * torch.randn(q0.shape, generator=g, dtype=torch.float64))
               for _ in range(T)]
    targets = [W.as_f32_exact(t.numpy()) for t in targets]
    scale = [0.05, 0.02, 0.02]
    hmin = torch.tensor(1e-3 * q0[:, 0].mean(axis=(1, 2)))
    loss_ref, g_ref, dq_ref = osn.loss_and_grads(q0, [torch.tensor(t) for t in targets], p, dt, hmin,
                                                 scale, round_bf16=True, want_dq0=True)
    net = gpu_net(fv, p)
    tape = fv.fv_tape_create(net, B, n, n, T, dt)
    fv.fv_tape_forward(tape, f32(q0).cuda())
    loss = fv.fv_tape_loss(tape, f32(np.stack(targets)).cuda(), scale)
    assert abs(loss - loss_ref) <= 1e-4 * abs(loss_ref), (loss, loss_ref)
    dparams = torch.zeros(fv.FV_NET_PARAMS, device="cuda")
    dq0 = fv.fv_tape_backward(tape, dparams, want_dq0=True)
    cos, rel = _cos_rel(dq0.cpu(), dq_ref)
    assert cos >= 0.9999 and rel <= 1e-2, ("dq0", cos, rel)
    gp = dparams.cpu().double()
    cos, rel = _cos_rel(gp, g_ref)
    assert cos >= 0.999 and rel <= 2e-2, ("dparams", cos, rel)
    if zero:
        nz = torch.nonzero(g_ref).reshape(-1)
        lo = 29796 - 36
        assert int(nz.min()) >= lo   # only b4


def test_tape_backward_replayed_from_a_graph_is_the_same(fv):
    """The first fv_tape_forward / fv_tape_backward of a tape runs its
    launches directly; later calls with the same buffers replay them from a
    captured CUDA graph.  The losses and gradients of the direct run, the
    capturing call and a replay agree bit for bit, and a call with another
    dq0 buffer is captured anew."""
    p = rand_params(6, last_scale=0.1)
    n, T, B, dt = 64, 3, 2, 1e-3
    q0 = swe_state(n, 21, members=B)
    g = torch.Generator().manual_seed(3)
    targets = np.stack([W.as_f32_exact((torch.tensor(q0) * (1 + 0.01 * torch.randn(q0.shape, generator=g,
                                                                                 dtype=torch.float64))).numpy())
                        for _ in range(T)])
    net = gpu_net(fv, p)
    tape = fv.fv_tape_create(net, B, n, n, T, dt)
    # the forward likewise: direct, capture + launch, replay (same snaps buffer)
    losses = []
    for _ in range(3):
        fv.fv_tape_forward(tape, f32(q0).cuda(), want_snaps=False)
        losses.append(fv.fv_tape_loss(tape, f32(targets).cuda(), [0.05, 0.02, 0.02]))
    assert losses[0] == losses[1] == losses[2], losses
    grads = []
    d = torch.zeros(fv.FV_NET_PARAMS, device="cuda")
    for _ in range(3):                      # direct, capture + launch, replay
        d.zero_()
        fv.fv_tape_backward(tape, d)
        grads.append(d.clone())
    assert float(grads[0].abs().max()) > 0
    assert torch.equal(grads[0], grads[1]) and torch.equal(grads[0], grads[2])
    d = torch.zeros(fv.FV_NET_PARAMS, device="cuda")
    dq_a = fv.fv_tape_backward(tape, d, want_dq0=True)
    d2 = torch.zeros(fv.FV_NET_PARAMS, device="cuda")
    dq_b = fv.fv_tape_backward(tape, d2, want_dq0=True)
    assert torch.equal(d, grads[0]) and torch.equal(d2, grads[0]) and torch.equal(dq_a, dq_b)


@pytest.mark.parametrize("ny,nx", [(16, 128), (64, 64)])
def test_stencil_net_backward_matches_oracle(fv, ny, nx):
    """stencil_net_backward (the network's VJP at q) against the oracle's FP64
    reverse mode through the BF16-mirrored forward and the normalisation, on
    a tile-mode grid and on the 64^2 training grid (several rows per tile).
    dparams and dq start from a known non-zero fill: the call adds to them."""
    p = rand_params(8, last_scale=0.3)
    net = gpu_net(fv, p)
    q0 = W.as_f32_exact(W.random_smooth_swe(nx, seed=5, members=2, vel=0.2)[:, :, :ny, :])
    g = torch.Generator().manual_seed(2)
    dw = torch.randn(2, 36, ny, nx, generator=g, dtype=torch.float64)
    flat = p.flat().clone().requires_grad_(True)
    W_, b_, off = [], [], 0
    for co, ci in osn.LAYER_SHAPES:
        n = co * ci * 9
        W_.append(flat[off:off + n].reshape(co, ci, 3, 3))
        off += n
        b_.append(flat[off:off + co])
        off += co
    q = torch.tensor(q0).requires_grad_(True)
    w = osn.normalise(osn.net_raw(q, osn.NetParams(W_, b_, p.mean, p.std), round_bf16=True))
    (w * dw).sum().backward()
    fill_p = torch.linspace(-1.0, 1.0, fv.FV_NET_PARAMS, device="cuda")
    fill_q = torch.full((2, 3, ny, nx), 0.75, device="cuda")
    dparams, dq = fv.net_backward(net, f32(q0).cuda(), f32(dw).cuda(), dparams=fill_p.clone(),
                                  dq=fill_q.clone())
    for got, fill, ref, name in ((dparams, fill_p, flat.grad, "dparams"), (dq, fill_q, q.grad, "dq")):
        a, b = (got - fill).double().cpu().reshape(-1), ref.reshape(-1)
        cos = float(a @ b / (a.norm() * b.norm()))
        rel = float((a - b).norm() / b.norm())
        assert cos >= 0.999 and rel <= 2e-2, (name, cos, rel)


@pytest.mark.parametrize("ny,nx", [(64, 64), (32, 256)])
def test_stencil_net_backward_is_deterministic(fv, ny, nx):
    """The weight gradients are reduced in a fixed order (per-CTA partial sums
    over fixed cell ranges, added in CTA order): two calls agree bit for bit."""
    p = rand_params(8, last_scale=0.3)
    net = gpu_net(fv, p)
    q0 = W.as_f32_exact(W.random_smooth_swe(nx, seed=5, members=3, vel=0.2)[:, :, :ny, :])
    g = torch.Generator().manual_seed(4)
    dw = torch.randn(3, 36, ny, nx, generator=g).float().cuda()
    a = fv.net_backward(net, f32(q0).cuda(), dw)
    b = fv.net_backward(net, f32(q0).cuda(), dw)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert float(a[0].abs().max()) > 0


@pytest.mark.parametrize("ny,nx,B", [(64, 64, 64), (256, 256, 16)])
def test_batched_convolutions_equal_single_members(fv, ny, nx, B):
    """A batch of many tiles runs the persistent convolution (weights resident
    per CTA, two staging buffers and accumulators); one member alone runs one
    tile per CTA.  Both issue each tile's MMAs in the same order, so the
    forward outputs of both networks and the backward's dq agree bit for
    bit, member by member."""
    from oracle import face_net as ofn
    p = rand_params(8, last_scale=0.3)
    net = gpu_net(fv, p)
    pf = ofn.init_params(3, MEAN, STD, scale=0.5)
    fnet = fv.face_net_create(pf.flat().numpy().astype(np.float32), MEAN, STD)
    q = f32(W.as_f32_exact(W.random_smooth_swe(nx, seed=7, members=B, vel=0.2)[:, :, :ny, :])).cuda()
    g = torch.Generator().manual_seed(9)
    dw = torch.randn(B, 36, ny, nx, generator=g).float().cuda()
    w_all = fv.stencil_net_forward(net, q)
    s_all = fv.face_net_forward(fnet, q)
    ds = dw[:, :12].contiguous()
    dq_all = fv.net_backward(net, q, dw)[1]
    dqf_all = fv.net_backward(fnet, q, ds)[1]
    for b in range(0, B, max(1, B // 8)):
        assert torch.equal(w_all[b:b + 1], fv.stencil_net_forward(net, q[b:b + 1])), b
        assert torch.equal(s_all[b:b + 1], fv.face_net_forward(fnet, q[b:b + 1])), b
        assert torch.equal(dq_all[b:b + 1], fv.net_backward(net, q[b:b + 1], dw[b:b + 1])[1]), b
        assert torch.equal(dqf_all[b:b + 1], fv.net_backward(fnet, q[b:b + 1], ds[b:b + 1])[1]), b
