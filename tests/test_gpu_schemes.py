"""Parity of the plain step with the other numerical fluxes (Lax-Friedrichs,
Rusanov, Roe, HLLE, HLLC; Eqs. 2.11-2.17) and with SSP-RK3 (Eq. 2.20) against
the FP64 oracle (``oracle.schemes``), through the C ABI, on both equations.
Tolerances follow the plain-step parity tests: max(fixed floor, 5 x the
oracle's own FP32-vs-FP64 roundoff on the same case), the latter measured
in the test."""
import numpy as np
import pytest
import torch

from helpers import f32, rel_errors
from oracle import fv as ofv
from oracle import schemes as S
from paper_2602_08670_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_O1 = (1e-5, 1e-4)          # depth, density, energy, O(1) momenta
TOL_SMALL = (1e-4, 2e-4)       # small momenta (O(1e-2)) after 100 steps
STEPS = 100


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv as binding
    return binding


def case(eq):
    if eq == ofv.SWE:
        q = W.swe_gaussian_bump(64, 48)
        q[:, 1] = 0.05 * np.sin(2 * np.pi * W.cell_centres(64))[None, None, :]
        q[:, 2] = 0.03 * np.cos(2 * np.pi * W.cell_centres(48))[None, :, None]
        return W.as_f32_exact(q), [TOL_O1, TOL_SMALL, TOL_SMALL]
    q = W.euler_kelvin_helmholtz(64, 64, seed=1)
    return W.as_f32_exact(q), [TOL_O1, TOL_O1, (2e-4, 3e-4), TOL_O1]


def gpu_replay(fv, q0, eq, dts, nsteps, flux, rk, variant="auto"):
    q0t = f32(q0).cuda()
    s = fv.swe_init(q0t, dt_mode="replay") if eq == ofv.SWE else fv.euler_init(q0t, dt_mode="replay")
    fv.fv_set_scheme(s, flux, rk)
    fv.fv_set_stage_variant(s, variant)
    fv.fv_set_replay_dt(s, dts)
    fv.fv_rollout(s, nsteps)
    return fv.fv_get_state(s).double().cpu(), s


def check(err, tols):
    for c, ((e2, ei), (l2, inf)) in enumerate(zip(err, tols)):
        assert e2 <= l2 and ei <= inf, (c, e2, ei, err)


def fp32_yardstick(q0, eq, dts, flux, rk, qr):
    """The oracle's own algorithm replayed in float32: its distance from the
    FP64 result is the roundoff the scheme amplifies on this case (large for
    Lax-Friedrichs, whose minmod faces and strong viscosity make it sensitive)."""
    q = torch.tensor(q0, dtype=torch.float32)
    dx, dy = ofv.grid_spacing(q)
    step = ofv.ssp_rk2 if rk == 2 else S.ssp_rk3
    for n in range(dts.shape[0]):
        dt = torch.tensor([float(dts[n, 0])], dtype=torch.float32)
        q = step(q, dt.view(1, 1, 1, 1), lambda s, dt=dt: S.rhs(s, eq, dx, dy, flux, dt))
    return rel_errors(q.double(), qr)


CASES = [(f, 2) for f in ("rusanov", "lf", "roe", "hlle", "hllc")] + \
        [(f, 3) for f in ("hll", "roe", "hllc")]


@pytest.mark.parametrize("eq", [ofv.SWE, ofv.EULER])
@pytest.mark.parametrize("flux,rk", CASES)
def test_scheme_matches_oracle(fv, flux, rk, eq):
    """Row-march kernels (nx = 64, a multiple of 4)."""
    q0, tols = case(eq)
    qr, tr, dts = S.run(torch.tensor(q0), eq, STEPS, flux=flux, rk=rk)
    q, s = gpu_replay(fv, q0, eq, dts[:, 0].numpy(), STEPS, flux, rk, "march")
    yard = fp32_yardstick(q0, eq, dts, flux, rk, qr)
    check(rel_errors(q, qr), [(max(l2, 5 * y2), max(li, 5 * yi)) for (l2, li), (y2, yi) in zip(tols, yard)])
    t, _, steps = fv.fv_get_time(s)
    assert steps[0] == STEPS and abs(t[0] - float(tr[0])) < 1e-12


@pytest.mark.parametrize("eq", [ofv.SWE, ofv.EULER])
@pytest.mark.parametrize("flux,rk", [("lf", 2), ("roe", 3), ("hllc", 3), ("hlle", 2)])
def test_tile_kernel_matches_oracle(fv, flux, rk, eq):
    """Shared-memory tile kernels: forced on nx = 64, and automatic on a
    ragged nx = 62 (not a multiple of 4) whose tiles leave a partial column."""
    q0, tols = case(eq)
    for q0c, variant in ((q0, "tile"), (np.ascontiguousarray(q0[..., :62]), "auto")):
        qr, tr, dts = S.run(torch.tensor(q0c), eq, 40, flux=flux, rk=rk)
        q, s = gpu_replay(fv, q0c, eq, dts[:, 0].numpy(), 40, flux, rk, variant)
        yard = fp32_yardstick(q0c, eq, dts, flux, rk, qr)
        check(rel_errors(q, qr), [(max(l2, 5 * y2), max(li, 5 * yi)) for (l2, li), (y2, yi) in zip(tols, yard)])


@pytest.mark.parametrize("eq", [ofv.SWE, ofv.EULER])
@pytest.mark.parametrize("ny,nx", [(12, 8), (6, 516)])
def test_march_edges_match_oracle(fv, eq, ny, nx):
    """Row-march kernels at the narrowest strip (nx = 8, wrap on both sides of
    one strip) and with a ragged last strip (nx = 516 = 512 + 4 columns), for
    Roe with SSP-RK2 and HLLC with SSP-RK3."""
    rng = np.random.default_rng(nx + ny)
    if eq == ofv.SWE:
        q0 = np.zeros((2, 3, ny, nx))
        q0[:, 0] = 1.0 + 0.1 * rng.random((2, ny, nx))
        q0[:, 1:] = 0.05 * rng.standard_normal((2, 2, ny, nx))
        tols = [TOL_O1, TOL_SMALL, TOL_SMALL]
    else:
        q0 = np.zeros((2, 4, ny, nx))
        q0[:, 0] = 1.0 + 0.2 * rng.random((2, ny, nx))
        q0[:, 1:3] = 0.1 * rng.standard_normal((2, 2, ny, nx))
        q0[:, 3] = 2.5 + 0.5 * (q0[:, 1] ** 2 + q0[:, 2] ** 2) / q0[:, 0]
        tols = [TOL_O1, TOL_SMALL, TOL_SMALL, TOL_O1]
    q0 = W.as_f32_exact(q0)
    for flux, rk in (("roe", 2), ("hllc", 3)):
        # member 0's adaptive dt sequence, replayed for both members
        _, _, dts = S.run(torch.tensor(q0[:1]), eq, 20, flux=flux, rk=rk)
        qr, _, dts = S.run(torch.tensor(q0), eq, 20, flux=flux, rk=rk, dt_mode=ofv.DT_REPLAY,
                           dts=dts[:, 0])
        q, _ = gpu_replay(fv, q0, eq, dts[:, 0].numpy(), 20, flux, rk, "march")
        yard = fp32_yardstick(q0, eq, dts, flux, rk, qr)
        check(rel_errors(q, qr), [(max(l2, 5 * y2), max(li, 5 * yi)) for (l2, li), (y2, yi) in zip(tols, yard)])


@pytest.mark.parametrize("flux", ["rusanov", "lf", "roe", "hlle", "hllc"])
def test_tile_and_march_agree(fv, flux):
    """Both kernels evaluate the same formulas per face and per cell: after
    a few steps they agree to a few FP32 ulps of the state."""
    q0, _ = case(ofv.EULER)
    _, _, dts = S.run(torch.tensor(q0), ofv.EULER, 5, flux=flux, rk=3)
    out = [gpu_replay(fv, q0, ofv.EULER, dts[:, 0].numpy(), 5, flux, 3, v)[0] for v in ("tile", "march")]
    scale = out[0].abs().amax(dim=(0, 2, 3), keepdim=True)
    assert ((out[0] - out[1]).abs() / scale).max() < 2e-5


def test_rk3_adaptive_dt_follows_the_oracle(fv):
    """Adaptive dt: the CFL reduction runs in the third stage; the GPU's dt
    sequence follows the oracle's to FP32 rounding of the wave speeds."""
    q0, tols = case(ofv.SWE)
    qr, tr, dts = S.run(torch.tensor(q0), ofv.SWE, 30, flux="hllc", rk=3)
    s = fv.swe_init(f32(q0).cuda())
    fv.fv_set_scheme(s, "hllc", 3)
    _, t = fv.fv_rollout(s, 30)
    assert abs(t[0] - float(tr[0])) <= 1e-5 * float(tr[0])
    check(rel_errors(fv.fv_get_state(s).double().cpu(), qr), tols)


def test_invalid_schemes_rejected(fv):
    s = fv.swe_init(torch.ones(1, 3, 16, 16, device="cuda"))
    with pytest.raises(fv.FvError):
        fv.fv_set_scheme(s, "hll", 4)
    fv.fv_set_scheme(s, "roe", 2)
    net = fv.stencil_net_create(None, [1.0, 0.0, 0.0], [1.0, 1.0, 1.0])
    with pytest.raises(fv.FvError) as ei:
        fv.fv_step(s, net=net)
    assert ei.value.code == fv.FV_EINVAL


def test_lake_at_rest_every_flux(fv):
    """A flat lake at rest is a fixed point of every flux and integrator."""
    q0 = torch.zeros(1, 3, 24, 40)
    q0[:, 0] = 1.25
    for flux in ("rusanov", "lf", "roe", "hlle", "hllc"):
        for rk in (2, 3):
            s = fv.swe_init(q0.cuda(), dt_mode="fixed", dt_fixed=1e-3)
            fv.fv_set_scheme(s, flux, rk)
            fv.fv_rollout(s, 20)
            assert torch.equal(fv.fv_get_state(s).cpu(), q0), (flux, rk)
