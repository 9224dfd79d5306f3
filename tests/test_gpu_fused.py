"""The fused learned stage kernel (CNN on tcgen05 + learned faces + HLL + RK in
one persistent kernel per stage) against the FP64 oracle and against the
two-pass path (CNN coefficients through device memory).  Grids cover one CTA
per row (nx = 128), clusters of 2, 4 and 8 CTAs exchanging halos through
distributed shared memory (nx = 256, 512, 1024), short row ranges that make
every member span several streams, and degenerate row counts."""
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


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv as binding
    return binding


def rand_params(seed, last_scale=0.1, scale=0.5):
    p = osn.init_params(seed, MEAN, STD, zero_last=False, scale=scale)
    p.W[3] = (p.W[3] * last_scale).to(torch.bfloat16).to(torch.float64)
    return p


def gpu_net(fv, p):
    return fv.stencil_net_create(p.flat().numpy().astype(np.float32), MEAN, STD)


def swe_state(ny, nx, seed, members):
    n = max(nx, ny)
    q = W.swe_random_bumps(n, seed, members)[:, :, :ny, :nx].copy()
    q[:, 1] = 0.02 * np.sin(np.arange(nx) * 2 * np.pi / nx)[None, None, :]
    q[:, 2] = 0.015 * np.cos(np.arange(ny) * 2 * np.pi / ny)[None, :, None]
    return W.as_f32_exact(q)


def run_gpu(fv, q0, net, steps, variant, dt=2e-4, dt_mode="fixed", hmin_frac=None):
    s = fv.swe_init(f32(q0).cuda(), dt_mode=dt_mode, dt_fixed=dt)
    fv.fv_set_learned_variant(s, variant)
    if hmin_frac is not None:
        fv.fv_set_learned_hmin(s, hmin_frac)
    fv.fv_rollout(s, steps, net=net)
    return s, fv.fv_get_state(s).double().cpu()


def oracle_rollout(q0, p, steps, dt, hmin_frac=1e-3):
    hmin = torch.tensor(hmin_frac * q0[:, 0].mean(axis=(1, 2)))
    q = torch.tensor(q0)
    for _ in range(steps):
        q = osn.learned_step(q, p, dt, hmin, round_bf16=True).detach()
    return q


def assert_close(q, ref, l2=1e-4, linf=1e-3):
    for c, (e2, ei) in enumerate(rel_errors(q, ref)):
        assert e2 < l2 and ei < linf, (c, e2, ei)


@pytest.mark.parametrize("ny,nx,B", [(128, 128, 2), (64, 256, 2), (32, 512, 1), (8, 1024, 1)])
def test_fused_matches_oracle(fv, ny, nx, B):
    """Against the BF16-mirrored FP64 oracle, up to the largest cluster (8 CTAs
    exchanging halos for a 1024-column row)."""
    p = rand_params(4)
    q0 = swe_state(ny, nx, 11, B)
    _, q = run_gpu(fv, q0, gpu_net(fv, p), 8, "fused")
    assert_close(q, oracle_rollout(q0, p, 8, 2e-4))


def test_fused_zero_network_is_first_order(fv):
    net = fv.stencil_net_create(None, MEAN, STD)
    q0 = swe_state(64, 256, 7, 2)
    _, q = run_gpu(fv, q0, net, 10, "fused")
    first = lambda Q, d, delta: ofv.first_order_faces(Q, d)
    qr, _, _, _ = ofv.run(torch.tensor(q0), ofv.SWE, 10, dt_mode=ofv.DT_FIXED, dt_fixed=2e-4, recon=first)
    assert_close(q, qr, 1e-5, 1e-4)


@pytest.mark.parametrize("ny,nx,B", [(128, 128, 3), (48, 256, 5), (16, 1024, 1), (3, 128, 1), (1, 256, 2)])
def test_fused_matches_two_pass(fv, ny, nx, B):
    """The two GPU paths agree to the BF16 rounding of the last layer's
    weights: the fused kernel evaluates the last layer in difference form
    (W[3s+j] - W[3s+2], rounded to BF16 once, Section 2.5.3's normalisation
    depends on r only through these differences), the two-pass path the 36
    raw outputs; each is as close to the oracle as the other (about 1e-5 in
    the momenta after 12 steps), so they agree to a few times that."""
    p = rand_params(8)
    net = gpu_net(fv, p)
    q0 = swe_state(ny, nx, 17, B)
    _, qf = run_gpu(fv, q0, net, 12, "fused")
    _, qt = run_gpu(fv, q0, net, 12, "two_pass")
    assert_close(qf, qt, 5e-5, 2e-4)


def test_fused_adaptive_dt_closes_every_member(fv):
    """Adaptive dt: each member's stage-2 reduction is closed once by the last
    of the streams that touch it (many streams per member here); time and dt
    follow the two-pass path."""
    p = rand_params(9)
    net = gpu_net(fv, p)
    q0 = swe_state(128, 128, 19, 7)
    sf, qf = run_gpu(fv, q0, net, 15, "fused", dt_mode="adaptive")
    st, qt = run_gpu(fv, q0, net, 15, "two_pass", dt_mode="adaptive")
    tf, dtf, nf = fv.fv_get_time(sf)
    tt, dtt, nt = fv.fv_get_time(st)
    assert list(nf) == [15] * 7 and list(nt) == [15] * 7
    assert np.allclose(tf, tt, rtol=1e-5) and np.allclose(dtf, dtt, rtol=1e-5)
    assert_close(qf, qt, 1e-5, 1e-4)
    assert list(fv.fv_health(sf)) == [0] * 7


def _fallback_margin(q0, p, steps, dt, frac):
    """Smallest distance, relative to h_min, between a learned face depth and
    h_min over both stages of every step of the oracle rollout, and the
    fraction of faces that fall back at the first stage."""
    hmin = torch.tensor(frac * q0[:, 0].mean(axis=(1, 2)))
    hm = hmin.view(-1, 1, 1)
    dx, dy = ofv.grid_spacing(torch.tensor(q0))
    q = torch.tensor(q0)
    margin, first = float("inf"), None
    for _ in range(steps):
        q1 = q + dt * osn.learned_rhs(q, p, dx, dy, hmin)
        for s in (q, q1):
            w = osn.normalise(osn.net_raw(s, p, True))
            for d, dim in ((0, -1), (1, -2)):
                QL, QR = osn.learned_faces(s, w, d, dim)
                for h in (QL[:, 0], QR[:, 0]):
                    margin = min(margin, float(((h - hm).abs() / hm).min()))
                if first is None:
                    first = float(((QL[:, 0] < hm) | (QR[:, 0] < hm)).double().mean())
        q = osn.learned_step(q, p, dt, hmin).detach()
    return margin, first


def test_fused_positivity_fallback_matches_oracle(fv):
    """Strongly extrapolating stencils with h_min just below the smallest
    depth, so that many faces fall back to minmod.  The fallback is a discrete
    choice taken in FP32 on the GPU and in FP64 in the oracle; h_min is picked
    so that no face depth comes within 2e-5 (relative) of it, where the two
    precisions could choose differently."""
    p = osn.init_params(0, MEAN, STD, zero_last=True)
    b4 = torch.zeros(36, dtype=torch.float64)
    for d in range(2):
        for v in range(3):
            b4[osn.out_channel(d, v, 0, 0)] = -6.0
            b4[osn.out_channel(d, v, 0, 2)] = 6.0
            b4[osn.out_channel(d, v, 1, 0)] = 6.0
            b4[osn.out_channel(d, v, 1, 2)] = -6.0
    p.b[3] = b4
    q0 = swe_state(16, 128, 2, 1)
    cands = [(_fallback_margin(q0, p, 3, 1e-4, f), f) for f in np.linspace(0.95, 0.999, 50)]
    (margin, share), frac = max((c for c in cands if c[0][1] > 0.01), key=lambda c: c[0][0])
    assert margin > 2e-5, (margin, share, frac)
    _, q = run_gpu(fv, q0, gpu_net(fv, p), 3, "fused", dt=1e-4, hmin_frac=frac)
    # FP32 rounding grows with the +-6 stencil weights: the 1e-4 bound of the
    # random-network comparisons (a single flipped fallback face costs ~1e-3)
    assert_close(q, oracle_rollout(q0, p, 3, 1e-4, hmin_frac=frac))


def test_fused_t_end_and_unsupported(fv):
    p = rand_params(10)
    net = gpu_net(fv, p)
    q0 = swe_state(128, 128, 23, 2)
    s = fv.swe_init(f32(q0).cuda(), dt_mode="fixed", dt_fixed=2e-4)
    fv.fv_set_learned_variant(s, "fused")
    fv.fv_rollout(s, 50, net=net, t_end=2.5 * 2e-4)
    t, _, n = fv.fv_get_time(s)
    assert np.allclose(t, 2.5 * 2e-4) and list(n) == [3, 3]
    s2 = fv.swe_init(torch.ones(1, 3, 64, 64, device="cuda"), dt_mode="fixed", dt_fixed=1e-4)
    with pytest.raises(fv.FvError) as ei:
        fv.fv_set_learned_variant(s2, "fused")
    assert ei.value.code == fv.FV_EINVAL
