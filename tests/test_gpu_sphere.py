"""Parity of shallow water on the sphere (Sections 2.4 and 4.3) with the FP64
oracle (``oracle.sphere``), through the C ABI: the device-computed grid
(centres, areas) against the oracle's, SSP-RK2 rollouts with the oracle's
adaptive dt replayed (tolerance max(floor, 5 x the oracle's own FP32 replay
distance), the lake at rest, mass conservation across the seams, and the
rejected settings."""
import numpy as np
import pytest
import torch

from helpers import f32, rel_errors
from oracle import sphere as S
from paper_2602_08670_gb300 import workloads as W

pytestmark = pytest.mark.gpu

G_ND = 11489.57      # g in Earth radii per day^2
OMEGA = 6.300388     # rotation rate in radians per day
FLOOR = [(1e-5, 1e-4)] + [(1e-4, 1e-3)] * 3


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv as binding
    return binding


def initial(G, seed, members, spin):
    """Bumps and a rigid rotation on the oracle's cell centres."""
    c = G.centre.permute(2, 0, 1).numpy()
    return W.as_f32_exact(W.sphere_bumps(c, seed, members, spin=spin))


@pytest.mark.parametrize("ny", [8, 25, 32])
def test_grid_matches_oracle(fv, ny):
    G = S.Grid(2 * ny, ny)
    s = fv.sphere_init(torch.ones(1, 4, ny, 2 * ny) * torch.tensor([1.0, 0, 0, 0]).view(1, 4, 1, 1),
                       g=G_ND, omega=OMEGA)
    c, a = fv.sphere_get_cells(s)
    assert np.abs(c - G.centre.permute(2, 0, 1).numpy()).max() < 2e-7
    assert np.abs(a / G.area.numpy() - 1).max() < 2e-6
    assert abs(a.astype(np.float64).sum() / (4 * np.pi) - 1) < 1e-6


@pytest.mark.parametrize("nx,ny,B,steps,spin", [(16, 8, 1, 20, 0.5), (64, 32, 2, 30, 0.5), (100, 50, 1, 20, 1.0),
                                                 (36, 18, 5, 15, 0.5)])
def test_rollout_matches_oracle(fv, nx, ny, B, steps, spin):
    """(16, 8): one partial tile; (100, 50): the thesis's coarsest grid, a
    ragged last tile in both directions; two members share the grid; five
    members (ragged 36 x 18) take the batched kernel that stages each tile's
    metrics once for all members."""
    G = S.Grid(nx, ny)
    q0 = initial(G, 4, B, spin)
    # member 0's adaptive dt sequence, replayed for every member
    _, tr, dts = S.run(torch.tensor(q0[:1]), G, steps, g=G_ND, omega=OMEGA)
    qr, _, _ = S.run(torch.tensor(q0), G, steps, g=G_ND, omega=OMEGA, dt_mode="replay", dts=dts[:, 0])
    q32, _, _ = S.run(torch.tensor(q0), G, steps, g=G_ND, omega=OMEGA, dt_mode="replay", dts=dts[:, 0],
                      dtype=torch.float32)
    s = fv.sphere_init(f32(q0).cuda(), g=G_ND, omega=OMEGA, dt_mode="replay")
    fv.fv_set_replay_dt(s, dts[:, 0].numpy())
    fv.fv_rollout(s, steps)
    q = fv.fv_get_state(s).double().cpu()
    assert float((qr - torch.tensor(q0)).abs().max()) > 1e-7      # it moved
    err = rel_errors(q, qr)
    yard = rel_errors(q32.double(), qr)
    for c, ((e2, ei), (l2, li), (y2, yi)) in enumerate(zip(err, FLOOR, yard)):
        assert e2 <= max(l2, 5 * y2) and ei <= max(li, 5 * yi), (c, err, yard)
    # the GPU's own adaptive dt follows the oracle's
    s2 = fv.sphere_init(f32(q0[:1]).cuda(), g=G_ND, omega=OMEGA)
    _, t = fv.fv_rollout(s2, steps)
    assert abs(t[0] - float(tr[0])) <= 1e-5 * float(tr[0])


@pytest.mark.parametrize("flux", ["rusanov", "roe", "hlle", "hllc"])
@pytest.mark.parametrize("nx,ny,B", [(64, 32, 1), (48, 24, 4)])
def test_fluxes_match_oracle(fv, flux, nx, ny, B):
    """Table 4's other fluxes on the sphere (tangential momenta passive), in
    the per-member kernel (one member) and the batched one (four)."""
    G = S.Grid(nx, ny)
    q0 = initial(G, 6, B, 0.7)
    _, _, dts = S.run(torch.tensor(q0[:1]), G, 15, g=G_ND, omega=OMEGA, flux=flux)
    qr, _, _ = S.run(torch.tensor(q0), G, 15, g=G_ND, omega=OMEGA, dt_mode="replay", dts=dts[:, 0], flux=flux)
    q32, _, _ = S.run(torch.tensor(q0), G, 15, g=G_ND, omega=OMEGA, dt_mode="replay", dts=dts[:, 0],
                      dtype=torch.float32, flux=flux)
    s = fv.sphere_init(f32(q0).cuda(), g=G_ND, omega=OMEGA, dt_mode="replay")
    fv.fv_set_scheme(s, flux, 2)
    fv.fv_set_replay_dt(s, dts[:, 0].numpy())
    fv.fv_rollout(s, 15)
    err = rel_errors(fv.fv_get_state(s).double().cpu(), qr)
    yard = rel_errors(q32.double(), qr)
    for c, ((e2, ei), (l2, li), (y2, yi)) in enumerate(zip(err, FLOOR, yard)):
        assert e2 <= max(l2, 5 * y2) and ei <= max(li, 5 * yi), (c, err, yard)


def test_lake_at_rest(fv):
    """Eq. 3.1's correction balances the pressure flux through edges whose
    normals do not close: a resting lake stays at rest to FP32 rounding."""
    ny = 32
    q0 = torch.zeros(1, 4, ny, 2 * ny)
    q0[:, 0] = 1.2e-3
    s = fv.sphere_init(q0.cuda(), g=G_ND, omega=OMEGA)
    fv.fv_rollout(s, 100)
    q = fv.fv_get_state(s).cpu().double()
    c = (G_ND * 1.2e-3) ** 0.5                            # gravity-wave speed
    assert float(q[:, 1:].abs().max()) / 1.2e-3 < 1e-5 * c
    assert float((q[:, 0] - 1.2e-3).abs().max()) < 1e-6 * 1.2e-3


def test_mass_conserved(fv):
    ny = 40
    s = fv.sphere_init(torch.ones(1, 4, ny, 2 * ny), g=G_ND, omega=OMEGA)
    c, a = fv.sphere_get_cells(s)
    q0 = W.as_f32_exact(W.sphere_bumps(c, 7, 1, spin=1.0))
    fv.fv_set_state(s, f32(q0).cuda())
    m0 = float((q0[0, 0] * a).sum())
    fv.fv_rollout(s, 300)
    q = fv.fv_get_state(s).cpu().double().numpy()
    assert abs(float((q[0, 0] * a).sum()) - m0) < 2e-6 * m0


def test_invalid_settings_rejected(fv):
    with pytest.raises(fv.FvError) as ei:
        fv.sphere_init(torch.ones(1, 4, 8, 8), g=G_ND, omega=OMEGA)          # nx != 2 ny
    assert ei.value.code == fv.FV_EINVAL
    s = fv.sphere_init(torch.ones(1, 4, 8, 16), g=G_ND, omega=OMEGA)
    for call in (lambda: fv.fv_set_scheme(s, "lf", 2), lambda: fv.fv_set_scheme(s, "hll", 3),
                 lambda: fv.fv_set_boundary(s, "wall"),
                 lambda: fv.fv_diagnostics(s),
                 lambda: fv.fv_step(s, net=fv.stencil_net_create(None, [1, 0, 0], [1, 1, 1]))):
        with pytest.raises(fv.FvError) as ei:
            call()
        assert ei.value.code == fv.FV_EINVAL
