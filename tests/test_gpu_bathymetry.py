"""Parity of the bed-slope source (Eq. 2.3) and of reflecting walls (Section
4.2) on the GPU against the FP64 oracle (``oracle.bathymetry``), through the
C ABI, for both stage kernels (row march where nx is a multiple of 4, the
shared-memory tile kernel everywhere).  The oracle's adaptive dt sequence is replayed on the GPU; tolerances
are max(fixed floor, 5 x the oracle's own FP32-vs-FP64 distance on the same
case), the latter measured in the test by replaying the oracle in float32."""
import numpy as np
import pytest
import torch

from helpers import f32, rel_errors
from oracle import bathymetry as OB
from oracle import fv as ofv
from paper_2602_08670_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_O1 = (1e-5, 1e-4)          # depth, density, energy
TOL_MOM = (1e-4, 2e-4)         # momenta


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv as binding
    return binding


def swe_case(nx, ny, bed, seed=3):
    z = W.as_f32_exact(W.perlin_bed(nx, ny, seed)) if bed else None
    q0 = W.swe_bump_over_bed(z) if bed else W.swe_gaussian_bump(nx, ny)
    # a cross-wall stream so that both walls reflect momentum, not only waves
    q0[:, 1] += 0.1 * q0[:, 0]
    q0[:, 2] -= 0.05 * q0[:, 0]
    return W.as_f32_exact(q0), z


def euler_case(nx, ny):
    return W.as_f32_exact(W.euler_kelvin_helmholtz(nx, ny, seed=2)), None


def gpu_run(fv, q0, eq, z, bc, flux, rk, dts, variant="auto"):
    q0t = f32(q0).cuda()
    s = fv.swe_init(q0t, dt_mode="replay") if eq == ofv.SWE else fv.euler_init(q0t, dt_mode="replay")
    fv.fv_set_scheme(s, flux, rk)
    fv.fv_set_stage_variant(s, variant)
    fv.fv_set_boundary(s, bc)
    if z is not None:
        fv.fv_set_bathymetry(s, torch.tensor(z, dtype=torch.float32))
    fv.fv_set_replay_dt(s, dts)
    fv.fv_rollout(s, len(dts))
    return fv.fv_get_state(s).double().cpu(), s


CASES = [
    # eq, nx, ny, bed, bc, flux, rk, steps
    (ofv.SWE, 64, 48, False, OB.WALL, "hll", 2, 80),
    (ofv.SWE, 64, 48, True, OB.PERIODIC, "roe", 2, 80),
    (ofv.SWE, 64, 48, True, OB.WALL, "roe", 2, 80),        # Section 4.2's configuration
    (ofv.SWE, 62, 37, True, OB.WALL, "hllc", 3, 60),       # ragged tiles on both axes
    (ofv.SWE, 20, 9, True, OB.WALL, "lf", 2, 40),          # one partial tile, shorter than a tile
    (ofv.SWE, 2, 2, True, OB.WALL, "hll", 2, 10),          # the smallest grid walls accept
    (ofv.SWE, 8, 12, True, OB.WALL, "roe", 2, 30),         # march: one strip, both walls in it
    (ofv.SWE, 516, 6, True, OB.WALL, "hllc", 3, 20),       # march: 4-column last strip at the east wall
    (ofv.SWE, 1024, 40, True, OB.WALL, "roe", 2, 20),      # march: two strips, several row blocks
    (ofv.SWE, 64, 2, True, OB.WALL, "roe", 2, 20),         # two rows: every y ghost is a mirror
    (ofv.EULER, 64, 64, False, OB.WALL, "hllc", 3, 60),
    (ofv.EULER, 62, 40, False, OB.WALL, "hlle", 2, 60),
    (ofv.EULER, 516, 12, False, OB.WALL, "rusanov", 2, 20),
]


def variants(nx):
    return ("tile", "march") if nx % 4 == 0 and nx >= 8 else ("auto",)


@pytest.mark.parametrize("eq,nx,ny,bed,bc,flux,rk,steps", CASES)
def test_matches_oracle(fv, eq, nx, ny, bed, bc, flux, rk, steps):
    q0, z = swe_case(nx, ny, bed) if eq == ofv.SWE else euler_case(nx, ny)
    zt = None if z is None else torch.tensor(z)
    qr, tr, dts = OB.run(torch.tensor(q0), steps, flux=flux, rk=rk, z=zt, bc=bc, eq=eq)
    q32, _, _ = OB.run(torch.tensor(q0), steps, flux=flux, rk=rk, z=zt, bc=bc, eq=eq,
                       dt_mode=ofv.DT_REPLAY, dts=dts[:, 0], dtype=torch.float32)
    yard = rel_errors(q32.double(), qr)
    tols = [TOL_O1, TOL_MOM, TOL_MOM] + ([TOL_O1] if eq == ofv.EULER else [])
    for variant in variants(nx):
        q, s = gpu_run(fv, q0, eq, z, bc, flux, rk, dts[:, 0].numpy(), variant)
        err = rel_errors(q, qr)
        for c, ((e2, ei), (l2, li), (y2, yi)) in enumerate(zip(err, tols, yard)):
            assert e2 <= max(l2, 5 * y2) and ei <= max(li, 5 * yi), (variant, c, err, yard)
        t, _, n = fv.fv_get_time(s)
        assert n[0] == steps and abs(t[0] - float(tr[0])) < 1e-9


@pytest.mark.parametrize("flux", ["rusanov", "roe", "hll", "hlle"])
def test_four_quadrant_riemann_matches_oracle(fv, flux):
    """Section 4.2's planar Euler test (a four-quadrant Riemann problem
    between walls, the fluxes of its tables) on seeded quadrant states."""
    q0 = W.as_f32_exact(W.euler_four_quadrant(64, 64, seed=4))
    qr, tr, dts = OB.run(torch.tensor(q0), 60, flux=flux, rk=2, bc=OB.WALL, eq=ofv.EULER)
    q32, _, _ = OB.run(torch.tensor(q0), 60, flux=flux, rk=2, bc=OB.WALL, eq=ofv.EULER,
                       dt_mode=ofv.DT_REPLAY, dts=dts[:, 0], dtype=torch.float32)
    yard = rel_errors(q32.double(), qr)
    for variant in ("tile", "march"):
        q, _ = gpu_run(fv, q0, ofv.EULER, None, OB.WALL, flux, 2, dts[:, 0].numpy(), variant)
        err = rel_errors(q, qr)
        for c, ((e2, ei), (y2, yi)) in enumerate(zip(err, yard)):
            l2, li = TOL_O1 if c in (0, 3) else TOL_MOM
            assert e2 <= max(l2, 5 * y2) and ei <= max(li, 5 * yi), (variant, c, err, yard)


@pytest.mark.parametrize("variant", ["tile", "march"])
@pytest.mark.parametrize("axis", ["x", "y"])
def test_lake_at_rest_on_a_linear_bed(fv, axis, variant):
    """A flat surface over a bed linear along one axis, between walls: one
    step leaves the interior at rest up to FP32 rounding of the pressure
    flux (the centred bed slope cancels the pressure-flux difference); the
    same state without the bed accelerates by g h dz/dx.  The two cells next
    to a wall are not balanced (the mirrored bed is flat there) and each of
    the two SSP-RK2 stages carries that two cells further, so the check
    starts four cells from the walls."""
    n = 32
    c = (np.arange(n) + 0.5) / n
    z1 = 0.25 * c - 0.125                       # exact in FP32, as is 1 - z
    z = np.tile(z1, (n, 1)) if axis == "x" else np.tile(z1[:, None], (1, n))
    q0 = torch.zeros(1, 3, n, n)
    q0[:, 0] = torch.tensor(1.0 - z, dtype=torch.float32)
    dt = 1e-3
    scale = 9.81 * 1.0 * 0.25 * dt               # |momentum| after one step without the source
    k = 1 if axis == "x" else 2
    out = []
    for bed in (True, False):
        s = fv.swe_init(q0.cuda(), dt_mode="fixed", dt_fixed=dt)
        fv.fv_set_scheme(s, "roe", 2)
        fv.fv_set_stage_variant(s, variant)
        fv.fv_set_boundary(s, "wall")
        if bed:
            fv.fv_set_bathymetry(s, torch.tensor(z, dtype=torch.float32).cuda())
        fv.fv_step(s)
        out.append(fv.fv_get_state(s).double().cpu()[0, k, 4:-4, 4:-4].abs())
    assert float(out[0].max()) < 1e-4 * scale, float(out[0].max())
    assert float(out[1].min()) > 0.5 * scale


@pytest.mark.parametrize("variant", ["tile", "march"])
def test_walls_conserve_mass_over_a_bed(fv, variant):
    """No mass crosses a wall: over a Perlin bed with an adaptive dt the
    total depth changes only by FP32 rounding of the cell updates."""
    q0, z = swe_case(48, 48, True, seed=7)
    s = fv.swe_init(f32(q0).cuda())
    fv.fv_set_scheme(s, "roe", 2)
    fv.fv_set_stage_variant(s, variant)
    fv.fv_set_boundary(s, "wall")
    fv.fv_set_bathymetry(s, torch.tensor(z, dtype=torch.float32))
    fv.fv_rollout(s, 300)
    m0 = float(f32(q0)[:, 0].double().sum())
    m = float(fv.fv_get_state(s).double()[:, 0].sum())
    assert abs(m - m0) < 2e-6 * m0, (m, m0)


def test_tile_and_march_agree(fv):
    """Walls and bed in both kernels: the same per-face and per-cell formulas,
    so after a few steps they agree to a few FP32 ulps of the state."""
    q0, z = swe_case(128, 40, True, seed=5)
    _, _, dts = OB.run(torch.tensor(q0), 5, flux="hllc", rk=3, z=torch.tensor(z), bc=OB.WALL)
    out = [gpu_run(fv, q0, ofv.SWE, z, OB.WALL, "hllc", 3, dts[:, 0].numpy(), v)[0] for v in ("tile", "march")]
    scale = out[0].abs().amax(dim=(0, 2, 3), keepdim=True)
    assert ((out[0] - out[1]).abs() / scale).max() < 2e-5


def test_clearing_restores_the_periodic_flat_step(fv):
    """Back to periodic with the bed cleared, the state follows the row-march
    path of the plain periodic scheme bit for bit."""
    q0, z = swe_case(64, 32, True)
    outs = []
    for set_then_clear in (True, False):
        s = fv.swe_init(f32(q0).cuda(), dt_mode="fixed", dt_fixed=2e-4)
        fv.fv_set_scheme(s, "roe", 2)
        if set_then_clear:
            fv.fv_set_boundary(s, "wall")
            fv.fv_set_bathymetry(s, torch.tensor(z, dtype=torch.float32))
            fv.fv_step(s)
            fv.fv_set_state(s, f32(q0).cuda())
            fv.fv_set_boundary(s, "periodic")
            fv.fv_set_bathymetry(s, None)
        fv.fv_rollout(s, 5)
        outs.append(fv.fv_get_state(s).cpu())
    assert torch.equal(outs[0], outs[1])


def test_invalid_configurations_rejected(fv):
    q = torch.ones(1, 3, 16, 16, device="cuda")
    z = torch.zeros(16, 16)
    e = fv.euler_init(torch.ones(1, 4, 16, 16, device="cuda") * torch.tensor([1.0, 0, 0, 2.5], device="cuda")
                      .view(1, 4, 1, 1))
    with pytest.raises(fv.FvError) as ei:
        fv.fv_set_bathymetry(e, z)                # a bed is a shallow-water term
    assert ei.value.code == fv.FV_EINVAL
    sq = fv.swe_init(q)
    with pytest.raises(fv.FvError) as ei:
        fv._check(fv.lib().fv_set_boundary(sq.handle, 7))
    assert ei.value.code == fv.FV_EINVAL
    thin = fv.swe_init(torch.ones(1, 3, 1, 16, device="cuda"))
    with pytest.raises(fv.FvError) as ei:
        fv.fv_set_boundary(thin, "wall")          # the mirror needs two cells per axis
    assert ei.value.code == fv.FV_EINVAL
    with pytest.raises(ValueError):
        fv.fv_set_bathymetry(sq, torch.zeros(8, 16))
    net = fv.stencil_net_create(None, [1.0, 0.0, 0.0], [1.0, 1.0, 1.0])
    for setup in (lambda s: fv.fv_set_boundary(s, "wall"),
                  lambda s: fv.fv_set_bathymetry(s, torch.zeros(32, 128))):
        s = fv.swe_init(torch.ones(1, 3, 32, 128, device="cuda"))
        setup(s)
        with pytest.raises(fv.FvError) as ei:
            fv.fv_step(s, net=net)                # the learned step is periodic and flat
        assert ei.value.code == fv.FV_EINVAL
