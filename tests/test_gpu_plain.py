"""Parity of the CUDA plain step (MUSCL-minmod + HLL + SSP-RK2) with the FP64
oracle, invariants on the GPU, and the full-size launch configuration checked
on sampled cells.  Calls go through the C ABI (Python binding)."""
import math

import numpy as np
import pytest
import torch

from helpers import f32, rel_errors
from oracle import fv as ofv
from paper_2602_08670_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# Tolerances (relative L2, relative Linf per variable).  The yardstick is the
# roundoff of the same algorithm in FP32: the oracle run in float32 against
# float64 on each case below gives, after 1000 steps of the 128^2 bump,
# 7e-7 / 2e-6 for h and 8e-5 / 9e-5 for hu, hv (momentum is a small quantity
# driven by differences of g h^2 / 2 with h ~ 1); after 300 steps of the KH
# case 3e-7..1e-6 for rho, rho u, E and 3e-5 / 5e-5 for rho v.  A GPU result
# must lie within max(1e-5 / 1e-4, 5 x yardstick) of the FP64 oracle.
TOL_H = (1e-5, 1e-4)          # depth, density, energy, O(1) momenta
TOL_MOM_SHORT = (1e-4, 1e-4)  # small momenta after <= 100 steps
TOL_KH_V = (2e-4, 3e-4)       # rho v of the KH layer after 300 steps


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv as binding
    return binding


def gpu_replay(fv, q0, eq, dts, nsteps):
    q0t = f32(q0).cuda()
    s = fv.swe_init(q0t, dt_mode="replay") if eq == ofv.SWE else fv.euler_init(q0t, dt_mode="replay")
    fv.fv_set_replay_dt(s, dts)
    fv.fv_rollout(s, nsteps)
    return fv.fv_get_state(s).double().cpu(), s


def check(err, tols):
    for c, ((e2, ei), (l2, inf)) in enumerate(zip(err, tols)):
        assert e2 <= l2 and ei <= inf, (c, e2, ei, err)


def fp32_replay(q0, eq, dts):
    """The oracle's own step replayed in float32 with the same dt sequence:
    its distance from the FP64 run is the roundoff this case amplifies."""
    q = torch.tensor(q0, dtype=torch.float32)
    dx, dy = ofv.grid_spacing(q)
    for n in range(dts.shape[0]):
        dt = torch.tensor([float(dts[n, 0])], dtype=torch.float32).view(1, 1, 1, 1)
        q = ofv.ssp_rk2(q, dt, lambda s: ofv.rhs(s, eq, dx, dy))
    return q.double()


def test_swe_bump_128_1000_steps_replay(fv):
    """The oracle workload: 128x128, Gaussian bump, CFL 0.5, 1000 steps.  The
    bar per variable is max(1e-5 / 1e-4, 5 x the FP32 yardstick) in relative
    L2 / Linf, the yardstick computed here from the oracle replayed in float32
    (about 7e-7 for the depth and 8e-5 for the momenta, which start at zero)."""
    q0 = W.as_f32_exact(W.swe_gaussian_bump(128, 128))
    qr, tr, dts, _ = ofv.run(torch.tensor(q0), ofv.SWE, 1000)
    q, s = gpu_replay(fv, q0, ofv.SWE, dts[:, 0].numpy(), 1000)
    err = rel_errors(q, qr)
    yard = rel_errors(fp32_replay(q0, ofv.SWE, dts), qr)
    for c, ((e2, ei), (y2, yi)) in enumerate(zip(err, yard)):
        assert e2 <= max(1e-5, 5 * y2) and ei <= max(1e-4, 5 * yi), (c, err, yard)
    assert yard[0][0] < 1e-5 and err[0][0] < 1e-5          # the depth meets the 1e-5 bar outright
    t, _, steps = fv.fv_get_time(s)
    assert steps[0] == 1000 and abs(t[0] - float(tr[0])) < 1e-12


def test_swe_bump_adaptive_dt_tracks_oracle(fv):
    q0 = W.as_f32_exact(W.swe_gaussian_bump(128, 128))
    qr, tr, dts, _ = ofv.run(torch.tensor(q0), ofv.SWE, 200)
    s = fv.swe_init(f32(q0).cuda(), cfl=0.5)
    _, t = fv.fv_rollout(s, 200)
    q = fv.fv_get_state(s).double().cpu()
    assert abs(t[0] - float(tr[0])) / float(tr[0]) < 1e-6
    # own dt from the FP32 Courant-rate reduction: 10x looser than replay
    check(rel_errors(q, qr), [(1e-4, 1e-3), (1e-3, 1e-3), (1e-3, 1e-3)])


@pytest.mark.parametrize("nx,ny,B", [(100, 70, 1), (13, 9, 2), (64, 16, 3), (130, 33, 1), (5, 200, 1)])
def test_swe_ragged_and_batched(fv, nx, ny, B):
    q0 = W.as_f32_exact(W.random_smooth_swe(max(nx, ny), seed=nx + ny, members=B, vel=0.2)[:, :, :ny, :nx])
    qr, _, dts, _ = ofv.run(torch.tensor(q0), ofv.SWE, 50, lx=nx / max(nx, ny), ly=ny / max(nx, ny))
    q0t = f32(q0).cuda()
    s = fv.swe_init(q0t, dt_mode="replay", lx=nx / max(nx, ny), ly=ny / max(nx, ny))
    fv.fv_set_replay_dt(s, dts[:, 0].numpy())   # members share the replayed dt
    qr2, _, _, _ = ofv.run(torch.tensor(q0), ofv.SWE, 50, dt_mode=ofv.DT_REPLAY, dts=dts[:, 0],
                           lx=nx / max(nx, ny), ly=ny / max(nx, ny))
    fv.fv_rollout(s, 50)
    q = fv.fv_get_state(s).double().cpu()
    check(rel_errors(q, qr2), [TOL_H, TOL_MOM_SHORT, TOL_MOM_SHORT])


def test_euler_kh_replay(fv):
    q0 = W.as_f32_exact(W.euler_kelvin_helmholtz(96, 96, seed=0))
    qr, _, dts, _ = ofv.run(torch.tensor(q0), ofv.EULER, 300)
    q, _ = gpu_replay(fv, q0, ofv.EULER, dts[:, 0].numpy(), 300)
    check(rel_errors(q, qr), [TOL_H, TOL_H, TOL_KH_V, TOL_H])


def test_euler_sod_y_direction(fv):
    q0 = W.as_f32_exact(W.euler_sod(4, 128, axis="y"))
    qr, _, dts, _ = ofv.run(torch.tensor(q0), ofv.EULER, 100)
    q, _ = gpu_replay(fv, q0, ofv.EULER, dts[:, 0].numpy(), 100)
    check(rel_errors(q, qr), [TOL_H] * 4)


def test_lake_at_rest_bitwise(fv):
    q0 = torch.zeros(2, 3, 40, 72)
    q0[:, 0] = 1.3
    s = fv.swe_init(q0.cuda())
    fv.fv_rollout(s, 50)
    assert torch.equal(fv.fv_get_state(s).cpu(), q0)


def test_conservation_fp64_sums(fv):
    q0 = W.as_f32_exact(W.random_smooth_swe(256, seed=11, vel=0.2))
    s = fv.swe_init(f32(q0).cuda())
    d0 = fv.fv_diagnostics(s)
    ref = ofv.diagnostics(torch.tensor(q0), ofv.SWE).numpy()
    assert np.allclose(d0, ref, rtol=1e-12, atol=1e-14)
    fv.fv_rollout(s, 500)
    d1 = fv.fv_diagnostics(s)
    scale = abs(d0[0, 0])
    assert np.abs(d1[0, :3] - d0[0, :3]).max() / scale < 1e-6


@pytest.mark.parametrize("shift", [(0, 64), (16, 0), (5, 7)])
def test_translation_invariance_bitwise(fv, shift):
    q0 = f32(W.random_smooth_swe(128, seed=2, vel=0.2))
    a = fv.swe_init(q0.cuda(), dt_mode="fixed", dt_fixed=2e-4)
    b = fv.swe_init(torch.roll(q0, shift, (-2, -1)).contiguous().cuda(), dt_mode="fixed", dt_fixed=2e-4)
    fv.fv_rollout(a, 20)
    fv.fv_rollout(b, 20)
    qa = fv.fv_get_state(a).cpu()
    qb = fv.fv_get_state(b).cpu()
    assert torch.equal(torch.roll(qa, shift, (-2, -1)), qb)


def test_transpose_symmetry(fv):
    """x <-> y with hu <-> hv commutes with the step: bitwise for the tile
    kernel (x and y faces go through one code path), to a few ulps for the
    row-march kernel (x and y faces are compiled at different code sites,
    where the SFU reciprocal may be scheduled differently)."""
    q0 = f32(W.random_smooth_swe(96, seed=4, vel=0.2))
    qt = q0.transpose(-1, -2)[:, [0, 2, 1]].contiguous()
    for variant in ("tile", "march"):
        a = fv.swe_init(q0.cuda(), dt_mode="fixed", dt_fixed=2e-4)
        b = fv.swe_init(qt.cuda(), dt_mode="fixed", dt_fixed=2e-4)
        fv.fv_set_stage_variant(a, variant)
        fv.fv_set_stage_variant(b, variant)
        fv.fv_rollout(a, 10)
        fv.fv_rollout(b, 10)
        qa = fv.fv_get_state(a).cpu().transpose(-1, -2)[:, [0, 2, 1]]
        qb = fv.fv_get_state(b).cpu()
        if variant == "tile":
            assert torch.equal(qa, qb)
        else:
            assert float((qa - qb).abs().max()) <= 4 * 1.2e-7 * float(qa.abs().max())


@pytest.mark.parametrize("eq,nx,ny,B", [(ofv.SWE, 576, 100, 1), (ofv.SWE, 1024, 77, 2),
                                        (ofv.SWE, 8, 8, 3), (ofv.EULER, 520, 40, 2),
                                        (ofv.SWE, 2048, 9, 1)])
def test_stage_variants_agree(fv, eq, nx, ny, B):
    """Row-march kernel (strips of 512 columns, ring-buffered rows, packed
    FP32x2 arithmetic) and tile kernel (64x16 shared-memory tiles, scalar)
    evaluate the same per-face formulas: after 20 steps they agree to a few
    ulps, including partial strips, short columns and batches."""
    if eq == ofv.SWE:
        q0 = f32(W.random_smooth_swe(max(nx, ny), seed=nx, members=B, vel=0.2)[:, :, :ny, :nx])
        init = lambda q: fv.swe_init(q.cuda(), dt_mode="fixed", dt_fixed=1e-4)
    else:
        q0 = f32(np.concatenate([W.euler_kelvin_helmholtz(nx, ny, seed=k) for k in range(B)]))
        init = lambda q: fv.euler_init(q.cuda(), dt_mode="fixed", dt_fixed=1e-4)
    outs = []
    for variant in ("tile", "march"):
        s = init(q0)
        fv.fv_set_stage_variant(s, variant)
        fv.fv_rollout(s, 20)
        outs.append(fv.fv_get_state(s).cpu())
    # ulp-level differences of the depth / density drive the momenta through
    # the pressure term, so all variables are held to a few tens of ulps of
    # the largest first-variable magnitude
    scale = float(outs[0][:, 0].abs().max())
    diff = (outs[0] - outs[1]).abs().amax(dim=(0, 2, 3))
    assert bool((diff <= 32 * 1.2e-7 * scale).all()), (diff, scale)


def test_t_end_stops_exactly(fv):
    q0 = W.as_f32_exact(W.swe_gaussian_bump(64, 64))
    s = fv.swe_init(f32(q0).cuda())
    _, t = fv.fv_rollout(s, 1000, t_end=0.05)
    assert t[0] == pytest.approx(0.05, abs=1e-15)
    _, _, steps = fv.fv_get_time(s)
    assert 0 < steps[0] < 1000
    _, t2 = fv.fv_rollout(s, 10, t_end=0.05)     # nothing left to do
    assert t2[0] == t[0]
    _, _, steps2 = fv.fv_get_time(s)
    assert steps2[0] == steps[0]


def test_snapshots_and_host_io(fv):
    q0 = f32(W.swe_gaussian_bump(64, 48))
    s = fv.swe_init(q0)                       # from host memory
    snaps, _ = fv.fv_rollout(s, 12, snap_every=4, snaps_on_device=False)
    assert snaps.shape == (3, 1, 3, 48, 64) and not snaps.is_cuda
    last = fv.fv_get_state(s, device=False)
    assert torch.equal(snaps[-1], last)
    s2 = fv.swe_init(q0.cuda())
    for _ in range(12):
        fv.fv_step(s2)
    fv.fv_sync(s2)
    assert torch.equal(fv.fv_get_state(s2).cpu(), last)


def test_unstable_member_is_reported_and_isolated(fv):
    q0 = f32(W.random_smooth_swe(64, seed=3, members=3, vel=0.1))
    q0[1, 0, 10, 10] = float("nan")
    s = fv.swe_init(q0.cuda(), dt_mode="fixed", dt_fixed=1e-4)
    with pytest.raises(fv.FvError) as ei:
        fv.fv_rollout(s, 5)
    assert ei.value.code == fv.FV_EUNSTABLE
    h = fv.fv_health(s)
    assert h[1] != 0 and h[0] == 0 and h[2] == 0
    clean = fv.swe_init(q0[[0, 2]].contiguous().cuda(), dt_mode="fixed", dt_fixed=1e-4)
    fv.fv_rollout(clean, 5)
    q_all = torch.empty(3, 3, 64, 64, device="cuda")
    with pytest.raises(fv.FvError):
        fv.fv_get_state(s, out=q_all)
    assert torch.equal(q_all[[0, 2]].cpu(), fv.fv_get_state(clean).cpu())


def test_fixed_dt_cfl_violation_flagged(fv):
    q0 = f32(W.swe_gaussian_bump(32, 32))
    s = fv.swe_init(q0.cuda(), dt_mode="fixed", dt_fixed=0.1)
    with pytest.raises(fv.FvError) as ei:
        fv.fv_rollout(s, 1)
    assert ei.value.code == fv.FV_EUNSTABLE
    assert fv.fv_health(s)[0] & 4


def _patch_oracle_step(q_full, j, i, dt, eq, r=6):
    """One oracle step of cell (j, i) computed on the periodic (2r+1)^2 patch
    around it: the centre depends only on cells within 4 (two stages of a
    2-cell stencil), so r = 6 leaves a margin."""
    ny, nx = q_full.shape[-2:]
    jj = [(j + d) % ny for d in range(-r, r + 1)]
    ii = [(i + d) % nx for d in range(-r, r + 1)]
    patch = torch.tensor(q_full[:, :, jj][:, :, :, ii], dtype=torch.float64)
    dx = 1.0 / nx
    L = lambda s: ofv.rhs(s, eq, dx, 1.0 / ny)
    return ofv.ssp_rk2(patch, dt, L)[:, :, r, r]


@pytest.mark.parametrize("eq,n", [(ofv.SWE, 4096), (ofv.EULER, 2048)])
def test_full_size_sampled_cells(fv, eq, n):
    """Full-size workloads in the bench launch configuration: one step on the
    GPU, sampled cells recomputed by the oracle one by one."""
    if eq == ofv.SWE:
        q0 = W.swe_gaussian_bump(n, n)
        q0[0, 1] = 0.05 * np.sin(2 * math.pi * W.cell_centres(n))[None, :]
        s = fv.swe_init(f32(q0).cuda(), cfl=0.5)
    else:
        q0 = W.euler_kelvin_helmholtz(n, n, seed=0)
        s = fv.euler_init(f32(q0).cuda(), cfl=0.5)
    q0 = W.as_f32_exact(q0)
    _, dt, _ = fv.fv_get_time(s)
    fv.fv_step(s)
    q = fv.fv_get_state(s).cpu().numpy()
    rng = np.random.default_rng(0)
    pts = [(int(a), int(b)) for a, b in rng.integers(0, n, size=(24, 2))]
    pts += [(0, 0), (n - 1, n - 1), (n // 2, n // 2), (n // 4, 3), (n - 2, n // 2 + 1)]
    for j, i in pts:
        ref = _patch_oracle_step(q0, j, i, float(dt[0]), eq).numpy()[0]
        got = q[0, :, j, i]
        # one FP32 step: errors of a few ulps of each variable's group scale
        # (momentum components share the largest momentum magnitude)
        scale = np.abs(q0[0]).max(axis=(1, 2))
        scale[1:3] = scale[1:3].max()
        assert np.all(np.abs(got - ref) <= 2e-6 * scale), (j, i, got, ref)


@pytest.mark.parametrize("eq", [ofv.SWE, ofv.EULER])
def test_checkpoint_resume_is_bitwise(fv, eq):
    """Save after 12 adaptive steps, load into a fresh state, run 20 more:
    bitwise the state, time and step count of the uninterrupted run."""
    q0 = W.random_smooth_swe(64, seed=8, members=2, vel=0.2) if eq == ofv.SWE else \
        np.concatenate([W.euler_kelvin_helmholtz(64, 48, seed=k) for k in range(2)])
    init = fv.swe_init if eq == ofv.SWE else fv.euler_init
    a = init(f32(q0).cuda())
    fv.fv_rollout(a, 12)
    blob = fv.fv_checkpoint_save(a)
    fv.fv_rollout(a, 20)
    b = init(torch.ones_like(f32(q0)).cuda() if eq == ofv.SWE else f32(q0).cuda())
    fv.fv_checkpoint_load(b, blob)
    fv.fv_rollout(b, 20)
    assert torch.equal(fv.fv_get_state(a), fv.fv_get_state(b))
    ta, tb = fv.fv_get_time(a), fv.fv_get_time(b)
    assert all(np.array_equal(x, y) for x, y in zip(ta, tb))
    # a checkpoint of another shape is refused
    c = init(f32(q0[:1]).cuda())
    with pytest.raises(fv.FvError):
        fv.fv_checkpoint_load(c, blob)
