"""Parity of the face-state path (Section 2.5.3, third approach) with the FP64
oracle (``oracle.face_net``): the tcgen05 CNN forward with GeLU layers (raw
outputs and Softplus / de-normalised side states), the SSP-RK2 step with a
random network, the lake at rest, and the workspace shared with the stencil
path.  Calls go through the C ABI.

Step tolerances: max(floor, 5 x the oracle's own FP32-vs-FP64 distance on
the same case).  That distance is large in the momenta here (~1e-2 relative
after 10 steps): the depth outputs drive the pressure flux directly, so a
BF16 rounding of a hidden activation that flips between two precisions moves
the momentum far more than FP32 roundoff would.  The network itself is held
to the BF16-mirrored oracle output by output in the forward tests."""
import math
import time

import numpy as np
import pytest
import torch

from helpers import f32, rel_errors
from oracle import face_net as ofn
from paper_2602_08670_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MEAN = [1.05, 0.0, 0.0]
STD = [0.05, 0.02, 0.02]


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv as binding
    return binding


def rand_params(seed, last_scale=1.0, scale=0.5, h_bias=None):
    """Random network (BF16 weights); a small last layer and a depth bias of
    softplus^-1(h_bias) keep the side states near a resting depth."""
    p = ofn.init_params(seed, MEAN, STD, scale=scale)
    W4 = (p.W[3] * last_scale).to(torch.bfloat16).to(torch.float64)
    b4 = p.b[3].clone()
    if h_bias is not None:
        b4[0::3] += math.log(math.expm1(h_bias))
    return ofn.FaceNetParams(p.W[:3] + [W4], p.b[:3] + [ofn.f32(b4)], p.mean, p.std)


def gpu_net(fv, p):
    return fv.face_net_create(p.flat().numpy().astype(np.float32), MEAN, STD)


FLOOR = [(1e-5, 1e-4), (1e-4, 1e-3), (1e-4, 1e-3)]


def check_against_yardstick(q, qr, q32):
    yard = rel_errors(q32.double(), qr)
    err = rel_errors(q, qr)
    for c, ((e2, ei), (l2, li), (y2, yi)) in enumerate(zip(err, FLOOR, yard)):
        assert e2 <= max(l2, 5 * y2) and ei <= max(li, 5 * yi), (c, err, yard)


@pytest.mark.parametrize("ny,nx", [(64, 64), (16, 128), (32, 256), (16, 8), (5, 128), (6, 64)])
def test_cnn_raw_and_sides_match_oracle(fv, ny, nx):
    p = rand_params(1)
    net = gpu_net(fv, p)
    q0 = W.as_f32_exact(W.random_smooth_swe(max(nx, ny), seed=3, members=2, vel=0.2)[:, :, :ny, :nx])
    qg = f32(q0).cuda()
    raw = fv.face_net_forward(net, qg, raw=True).double().cpu()
    ref = ofn.net_raw(torch.tensor(q0), p, round_bf16=True).detach()
    scale = float(ref.abs().max())
    err = (raw - ref).abs()
    # BF16 activations on both sides; FP32 (GPU) vs FP64 (oracle) sums and
    # erf can flip a BF16 rounding now and then
    assert float(err.max()) <= 1e-2 * scale, (float(err.max()), scale)
    assert float(err.mean()) <= 1e-3 * scale, (float(err.mean()), scale)
    sides = fv.face_net_forward(net, qg).double().cpu()
    # the side-state epilogue applied to the GPU's own raw outputs (FP32
    # Softplus and de-normalisation against FP64)
    want = ofn.side_states(raw, p).reshape(sides.shape)
    assert torch.allclose(sides, want, rtol=2e-6, atol=1e-7)
    assert bool((sides[:, 0::3] > 0).all())


def test_zero_network_sides(fv):
    """All-zero weights: every side state is (ln 2, mean_hu, mean_hv)."""
    net = fv.face_net_create(None, [1.0, 0.25, -0.5], [1.0, 1.0, 1.0])
    s = fv.face_net_forward(net, torch.rand(1, 3, 16, 128, device="cuda") + 0.5).cpu()
    assert torch.allclose(s[:, 0::3], torch.full_like(s[:, 0::3], math.log(2.0)), rtol=1e-6, atol=0)
    assert torch.equal(s[:, 1::3], torch.full_like(s[:, 1::3], 0.25))
    assert torch.equal(s[:, 2::3], torch.full_like(s[:, 2::3], -0.5))


def test_step_random_network_matches_oracle(fv):
    p = rand_params(4, last_scale=0.1, h_bias=1.05)
    net = gpu_net(fv, p)
    q0 = W.as_f32_exact(W.swe_random_bumps(64, 11, 2))
    dt = 2e-4
    s = fv.swe_init(f32(q0).cuda(), dt_mode="fixed", dt_fixed=dt)
    fv.fv_rollout(s, 10, net=net)
    q = fv.fv_get_state(s).double().cpu()
    qr, _, _ = ofn.run(torch.tensor(q0), p, 10, dt_mode="fixed", dt_fixed=dt)
    q32, _, _ = ofn.run(torch.tensor(q0), p, 10, dt_mode="fixed", dt_fixed=dt, dtype=torch.float32)
    qr = qr.detach()
    assert float((qr - torch.tensor(q0)).abs().max()) > 1e-4    # the state did move
    check_against_yardstick(q, qr, q32)


def test_adaptive_step_follows_the_oracle(fv):
    """Adaptive dt (CFL 0.5 on the state at the start of each step): the
    oracle's dt sequence, replayed, and the GPU's own."""
    p = rand_params(5, last_scale=0.1, h_bias=1.05)
    net = gpu_net(fv, p)
    q0 = W.as_f32_exact(W.swe_random_bumps(128, 12, 1)[:, :, :32, :])
    qr, tr, dts = ofn.run(torch.tensor(q0), p, 6)
    q32, _, _ = ofn.run(torch.tensor(q0), p, 6, dt_mode="replay", dts=dts[:, 0], dtype=torch.float32)
    s = fv.swe_init(f32(q0).cuda(), dt_mode="replay")
    fv.fv_set_replay_dt(s, dts[:, 0].numpy())
    fv.fv_rollout(s, 6, net=net)
    check_against_yardstick(fv.fv_get_state(s).double().cpu(), qr.detach(), q32)
    s2 = fv.swe_init(f32(q0).cuda())
    _, t = fv.fv_rollout(s2, 6, net=net)
    assert abs(t[0] - float(tr[0])) <= 1e-5 * float(tr[0])


def test_lake_at_rest_is_kept_bitwise(fv):
    """A network that outputs the resting state on every side (zero weights,
    depth bias softplus^-1(h0)): equal states meet at every face, so the
    flux differences vanish and the lake stays bitwise at rest."""
    h0 = 1.25
    flat = np.zeros(fv.FV_FACE_NET_PARAMS, dtype=np.float32)
    flat[-12::3] = math.log(math.expm1(h0))
    net = fv.face_net_create(flat, [0, 0, 0], [1, 1, 1])
    sides = fv.face_net_forward(net, torch.full((1, 3, 16, 128), 0.0, device="cuda"))
    hs = float(sides[0, 0, 0, 0])
    q0 = torch.zeros(1, 3, 16, 128)
    q0[:, 0] = hs
    s = fv.swe_init(q0.cuda(), dt_mode="fixed", dt_fixed=1e-3)
    fv.fv_rollout(s, 20, net=net)
    assert torch.equal(fv.fv_get_state(s).cpu(), q0)


def test_face_then_stencil_network_on_one_state(fv):
    """The learned workspace serves both kinds: face-state steps, then
    stencil steps on the same state, match a state that took the stencil
    steps from the same starting point."""
    pf = rand_params(6, last_scale=0.1, h_bias=1.05)
    fnet = gpu_net(fv, pf)
    snet = fv.stencil_net_create(None, MEAN, STD)       # zero network: first-order scheme
    q0 = W.as_f32_exact(W.swe_random_bumps(128, 13, 1))
    s = fv.swe_init(f32(q0).cuda(), dt_mode="fixed", dt_fixed=1e-4)
    fv.fv_rollout(s, 3, net=fnet)
    mid = fv.fv_get_state(s).clone()
    fv.fv_rollout(s, 3, net=snet)
    s2 = fv.swe_init(mid, dt_mode="fixed", dt_fixed=1e-4)
    fv.fv_rollout(s2, 3, net=snet)
    assert torch.equal(fv.fv_get_state(s).cpu(), fv.fv_get_state(s2).cpu())


def test_kinds_are_checked(fv):
    fnet = fv.face_net_create(None, MEAN, STD)
    snet = fv.stencil_net_create(None, MEAN, STD)
    q = torch.ones(1, 3, 16, 128, device="cuda")
    assert fnet.kind == "face" and fnet.n_params == fv.FV_FACE_NET_PARAMS
    assert snet.kind == "stencil" and snet.n_params == fv.FV_NET_PARAMS
    for call in (lambda: fv.face_net_forward(snet, q), lambda: fv.stencil_net_forward(fnet, q),
                 lambda: fv.face_net_forward(fnet, torch.ones(1, 3, 100, 100, device="cuda"))):
        with pytest.raises(fv.FvError) as ei:
            call()
        assert ei.value.code == fv.FV_EINVAL
    got = fv.stencil_net_get_params(fnet)
    assert got.shape == (fv.FV_FACE_NET_PARAMS,) and not got.any()
    s = fv.swe_init(q)
    fv.fv_set_scheme(s, "roe", 2)
    with pytest.raises(fv.FvError) as ei:
        fv.fv_step(s, net=fnet)                   # HLL and SSP-RK2 only
    assert ei.value.code == fv.FV_EINVAL


def test_server_runs_face_state_requests(fv):
    """Learned requests on a server built with a face-state network give the
    result of fv_rollout with that network (same adaptive dt, bitwise)."""
    p = rand_params(7, last_scale=0.1, h_bias=1.05)
    net = gpu_net(fv, p)
    q0 = W.as_f32_exact(W.swe_random_bumps(128, 14, 1))[0].astype(np.float32)
    server = fv.fv_server_create(2 << 30, 2, net)
    t = fv.submit(server, q0, eq="swe", nsteps=12, learned=True, cfl=0.4)
    t0 = time.time()
    r = None
    while r is None:
        r = fv.poll(server, t)
        assert time.time() - t0 < 60
        time.sleep(0.001)
    s = fv.swe_init(torch.tensor(q0)[None].cuda(), cfl=0.4)
    fv.fv_rollout(s, 12, net=net)
    assert torch.equal(torch.as_tensor(r[0]).reshape(1, 3, 128, 128).cpu(), fv.fv_get_state(s).cpu())


def _cos_rel(a, b):
    a = torch.as_tensor(a, dtype=torch.float64).reshape(-1)
    b = torch.as_tensor(b, dtype=torch.float64).reshape(-1)
    return float(a @ b / (a.norm() * b.norm())), float((a - b).norm() / b.norm())


@pytest.mark.parametrize("n,T,B", [(16, 2, 2), (64, 3, 2)])
def test_rollout_gradients_match_oracle(fv, n, T, B):
    """Loss (Eq. 2.28) and its gradient w.r.t. the parameters and the initial
    state through a T-step face-state rollout: the hand-written backward
    (HLL VJP per face, Softplus' from the side depths, GeLU' from the stored
    BF16 pre-activations, tcgen05 dX, deterministic dW) against the oracle's
    FP64 reverse-mode gradient of the same BF16-mirrored forward."""
    p = rand_params(6, last_scale=0.1, h_bias=1.05)
    dt = 1e-3 if n == 64 else 2e-3
    q0 = W.as_f32_exact(W.swe_random_bumps(n, 21, B))
    g = torch.Generator().manual_seed(3)
    targets = [W.as_f32_exact((torch.tensor(q0) * (1 + 0.01 * torch.randn(q0.shape, generator=g,
                                                                           dtype=torch.float64))).numpy())
               for _ in range(T)]
    scale = [0.05, 0.02, 0.02]
    loss_ref, g_ref, dq_ref = ofn.loss_and_grads(q0, [torch.tensor(t) for t in targets], p, dt, scale,
                                                 round_bf16=True, want_dq0=True)
    net = gpu_net(fv, p)
    tape = fv.fv_tape_create(net, B, n, n, T, dt)
    fv.fv_tape_forward(tape, f32(q0).cuda())
    loss = fv.fv_tape_loss(tape, f32(np.stack(targets)).cuda(), scale)
    assert abs(loss - loss_ref) <= 1e-4 * abs(loss_ref), (loss, loss_ref)
    dparams = torch.zeros(fv.FV_FACE_NET_PARAMS, device="cuda")
    dq0 = fv.fv_tape_backward(tape, dparams, want_dq0=True)
    cos, rel = _cos_rel(dq0.cpu(), dq_ref)
    assert cos >= 0.9999 and rel <= 1e-2, ("dq0", cos, rel)
    cos, rel = _cos_rel(dparams.cpu().double(), g_ref)
    assert cos >= 0.999 and rel <= 2e-2, ("dparams", cos, rel)


def test_device_gelu_matches_the_definition(fv):
    """The GeLU of the hidden-layer epilogue against x Phi(x) in FP64, read
    through bias-only networks: with W2 = W3 = 0 the third layer's
    activations are BF16(GeLU(b3)) in every cell, and W4 copies channel k to
    output k.  The BF16 roundings must agree except where the value lies
    within the FP32 evaluation's error of a rounding boundary.  The sweep
    stops at x = -4: further out the relative accuracy of the epilogue's erf
    (Hastings' approximation, absolute error <= 3e-7) fades, where
    |GeLU| < 1e-4."""
    from oracle import face_net as ofn
    xs = np.concatenate([np.linspace(-4.0, 6.0, 589), [0.0, 1.0, -1.0, 0.5, -0.5, 3.0, -3.0, 1e-3, -1e-3, 20.0, 7.5]])
    xs = xs.astype(np.float32)
    layout = ofn.FaceNetParams.from_flat(torch.zeros(ofn.n_params(), dtype=torch.float64), MEAN, STD)
    sizes = [w.numel() + b.numel() for w, b in zip(layout.W, layout.b)]
    off3 = sizes[0] + sizes[1] + layout.W[2].numel()           # b3
    off4 = sum(sizes[:3])                                       # W4
    got = []
    for k0 in range(0, len(xs), 12):
        chunk = xs[k0:k0 + 12]
        flat = np.zeros(fv.FV_FACE_NET_PARAMS, dtype=np.float32)
        flat[off3:off3 + len(chunk)] = chunk
        for k in range(len(chunk)):
            flat[off4 + ((k * 32 + k) * 3 + 1) * 3 + 1] = 1.0   # W4[k][k][1][1]
        net = fv.face_net_create(flat, MEAN, STD)
        raw = fv.face_net_forward(net, torch.ones(1, 3, 16, 128, device="cuda"), raw=True)
        got.append(raw[0, :len(chunk), 3, 5].double().cpu().numpy())
    got = np.concatenate(got)
    x = torch.tensor(xs, dtype=torch.float64)
    exact = (0.5 * x * (1.0 + torch.erf(x / np.sqrt(2.0))))
    want = exact.to(torch.float32).to(torch.bfloat16).double().numpy()
    ulp = np.maximum(np.abs(want), 1e-30) * 2.0 ** -7
    assert np.all(np.abs(got - want) <= ulp), np.max(np.abs(got - want) / ulp)
    assert np.mean(got == want) >= 0.95, np.mean(got == want)


@pytest.mark.parametrize("ny,nx", [(16, 128), (64, 64)])
def test_face_net_backward_matches_oracle(fv, ny, nx):
    """face_net_backward (the network's VJP at q) against the oracle's FP64
    reverse mode through the BF16-mirrored forward and the side-state
    epilogue, on a tile-mode grid and on the 64^2 training grid; dparams and
    dq start from a known non-zero fill (the call adds to them)."""
    p = rand_params(9, last_scale=0.3, h_bias=1.05)
    net = gpu_net(fv, p)
    q0 = W.as_f32_exact(W.random_smooth_swe(nx, seed=6, members=2, vel=0.2)[:, :, :ny, :])
    g = torch.Generator().manual_seed(3)
    ds = torch.randn(2, 12, ny, nx, generator=g, dtype=torch.float64)
    flat = p.flat().detach().clone().requires_grad_(True)
    pp = ofn.FaceNetParams.from_flat(flat, p.mean, p.std)
    q = torch.tensor(q0).requires_grad_(True)
    sides = ofn.side_states(ofn.net_raw(q, pp, round_bf16=True), pp).reshape(2, 12, ny, nx)
    (sides * ds).sum().backward()
    fill_p = torch.linspace(-1.0, 1.0, fv.FV_FACE_NET_PARAMS, device="cuda")
    fill_q = torch.full((2, 3, ny, nx), -0.5, device="cuda")
    dparams, dq = fv.net_backward(net, f32(q0).cuda(), f32(ds).cuda(), dparams=fill_p.clone(),
                                  dq=fill_q.clone())
    for got, fill, ref, name in ((dparams, fill_p, flat.grad, "dparams"), (dq, fill_q, q.grad, "dq")):
        a, b = (got - fill).double().cpu().reshape(-1), ref.reshape(-1)
        cos = float(a @ b / (a.norm() * b.norm()))
        rel = float((a - b).norm() / b.norm())
        assert cos >= 0.999 and rel <= 2e-2, (name, cos, rel)
