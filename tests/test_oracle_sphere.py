"""Pins of the spherical shallow-water oracle (``oracle.sphere``, Sections 2.4
and 4.3): the mapped grid tiles the sphere exactly and its seams coincide,
the edge frames are orthonormal and oriented, a lake at rest is steady
(Eq. 3.1's correction), mass is conserved across the seams, the scheme is
equivariant under the grid's 90-degree rotation about the polar axis, an
inertial oscillation turns at the Coriolis rate of Eq. 3.2, and the scheme
converges on a smooth flow.  CPU only."""
import math

import numpy as np
import pytest
import torch

from oracle import sphere as S

G_ND = 11489.57      # g in Earth radii per day^2
OMEGA = 6.300388     # Earth's rotation rate in radians per day


def bump_state(G, seed, amp=2e-5, depth=1.2e-3, vel=0.0):
    """Seeded Gaussian height bumps on the sphere, optionally with a random
    tangent momentum field."""
    rng = np.random.default_rng(seed)
    x = G.centre
    h = torch.full(x.shape[:2], depth, dtype=torch.float64)
    for _ in range(3):
        c = torch.tensor(rng.normal(size=3))
        c = c / c.norm()
        h = h + amp * torch.exp(-((x - c) ** 2).sum(-1) / 0.15)
    q = torch.zeros(1, 4, *x.shape[:2], dtype=torch.float64)
    q[0, 0] = h
    if vel:
        w = torch.tensor(rng.normal(size=3))
        m = torch.cross(w.expand_as(x), x, dim=-1) * vel * h[..., None]     # a rigid rotation: tangent
        q[0, 1:] = m.permute(2, 0, 1)
    return q


@pytest.mark.parametrize("ny", [4, 16, 40])
def test_grid_tiles_the_sphere(ny):
    G = S.Grid(2 * ny, ny)
    assert abs(float(G.area.sum()) - 4 * math.pi) < 1e-13 * 4 * math.pi
    assert float(G.area.min()) > 0
    assert float((G.P.norm(dim=-1) - 1).abs().max()) < 1e-15
    # x is periodic (the equator at xc = -3 is the one at xc = 1), the top and
    # bottom edges are glued to themselves reversed, and xc = -1 is the equator
    assert torch.equal(G.P[:, 0], G.P[:, -1])
    assert torch.equal(G.P[-1], G.P[-1].flip(0)) and torch.equal(G.P[0], G.P[0].flip(0))
    # each square's rim is the equator, its interior the open hemisphere
    for col in (0, ny, 2 * ny):
        assert float(G.P[:, col, 2].abs().max()) == 0.0
    assert float(G.P[0, :, 2].abs().max()) == 0.0 and float(G.P[-1, :, 2].abs().max()) == 0.0
    assert bool((G.P[1:-1, ny + 1:-1, 2] > 0).all()) and bool((G.P[1:-1, 1:ny, 2] < 0).all())


def test_disk_mapping_special_points():
    """Section 2.4's mapping: the square's centre goes to the disk's centre,
    its rim onto the unit circle, its corners to the 45-degree points, and a
    vertical segment x_c = d onto an arc through (D, +-D) (D = d / sqrt 2)."""
    xc = torch.tensor([0.0, 1.0, 1.0, -1.0, 0.3, 1.0], dtype=torch.float64)
    yc = torch.tensor([0.0, 0.0, 1.0, 1.0, 1.0, -0.4], dtype=torch.float64)
    xp, yp, z2 = S.disk_map(xc, yc)
    r = 1 / math.sqrt(2)
    assert torch.allclose(torch.stack([xp, yp])[:, :4],
                          torch.tensor([[0, 1, r, -r], [0, 0, r, r]], dtype=torch.float64), atol=1e-15)
    assert float(z2[1:].abs().max()) < 1e-15          # the rim is the equator
    assert torch.allclose(xp ** 2 + yp ** 2 + z2, torch.ones_like(z2), atol=1e-15)
    d = 0.6
    ys = torch.linspace(-d, d, 7, dtype=torch.float64)
    xp, yp, _ = S.disk_map(torch.full_like(ys, d), ys)
    D = d / math.sqrt(2)
    assert torch.allclose(xp[[0, -1]], torch.full((2,), D, dtype=torch.float64), atol=1e-15)
    assert torch.allclose(yp[[0, -1]], torch.tensor([-D, D], dtype=torch.float64), atol=1e-15)
    x0 = D - math.sqrt(1 - D * D)                      # the arc's centre (x0, 0), radius 1
    assert torch.allclose((xp - x0) ** 2 + yp ** 2, torch.ones_like(xp), atol=1e-14)


def test_frames_orthonormal_and_oriented():
    G = S.Grid(24, 12)
    for n, t, r in ((G.fx_n, G.fx_t, G.fx_r), (G.fy_n, G.fy_t, G.fy_r)):
        for a, b in ((n, t), (n, r), (t, r)):
            assert float((a * b).sum(-1).abs().max()) < 1e-14
        for a in (n, t, r):
            assert float((a.norm(dim=-1) - 1).abs().max()) < 1e-14
    # x normals point from cell i - 1 to cell i
    assert bool((((G.centre - torch.roll(G.centre, 1, 1)) * G.fx_n).sum(-1) > 0).all())
    # a seam edge seen from its two cells: equal lengths, opposite normals
    assert torch.equal(G.fy_n[-1], -G.fy_n[-1].flip(0)) and torch.equal(G.fy_len[-1], G.fy_len[-1].flip(0))
    assert torch.equal(G.fy_n[0], -G.fy_n[0].flip(0))


FLUXES = ["hll", "rusanov", "roe", "hlle", "hllc"]


def test_passive_splitting_reproduces_the_four_variable_flux():
    """The other fluxes treat m.t and m.r as two passive variables by solving
    (h, m.n, m.t) and (h, m.n, m.r): for HLL, whose four-variable form is
    written out in ``hll4``, the split gives the same flux."""
    from oracle import fv as ofv
    from oracle import schemes as Sc
    g = torch.Generator().manual_seed(5)
    qL = torch.rand(3, 4, 7, generator=g, dtype=torch.float64) * 0.2 - 0.1
    qR = torch.rand(3, 4, 7, generator=g, dtype=torch.float64) * 0.2 - 0.1
    qL[:, 0] = 1.0 + qL[:, 0]
    qR[:, 0] = 1.0 + qR[:, 0]
    a = Sc.normal_flux_solver("hll", qL[:, :3], qR[:, :3], ofv.SWE, 9.81, 1.4)
    b = Sc.normal_flux_solver("hll", qL[:, [0, 1, 3]], qR[:, [0, 1, 3]], ofv.SWE, 9.81, 1.4)
    assert torch.equal(a[:, :2], b[:, :2])
    assert torch.allclose(torch.cat([a, b[:, 2:3]], 1), S.hll4(qL, qR, 9.81), rtol=0, atol=1e-15)


@pytest.mark.parametrize("flux", FLUXES)
def test_lake_at_rest_is_steady(flux):
    """Uniform depth, no motion: without Eq. 3.1's correction the pressure
    flux through edges whose normals do not close on the curved surface would
    drive a flow of order g h^2 / dx; with it the tendency is rounding."""
    G = S.Grid(32, 16)
    q = torch.zeros(1, 4, 16, 32, dtype=torch.float64)
    q[:, 0] = 1.2e-3
    L = S.rhs(q, G, G_ND, OMEGA, flux)
    scale = 0.5 * G_ND * 1.2e-3 ** 2 * float(G.perimeter.max() / G.area.min())
    assert float(L.abs().max()) < 1e-12 * scale
    q1, _, _ = S.run(q, G, 5, g=G_ND, omega=OMEGA, flux=flux)
    assert float((q1 - q).abs().max()) < 1e-16


@pytest.mark.parametrize("flux", FLUXES)
def test_mass_conserved_and_momentum_tangent(flux):
    G = S.Grid(40, 20)
    q0 = bump_state(G, 1, vel=0.05)
    m0 = float(S.mass(q0, G))
    q, _, _ = S.run(q0, G, 30, g=G_ND, omega=OMEGA, flux=flux)
    assert abs(float(S.mass(q, G)) - m0) < 1e-13 * m0
    x = G.centre.permute(2, 0, 1)
    assert float((q[0, 1:] * x).sum(0).abs().max()) < 1e-18
    assert float((q - q0).abs().max()) > 1e-7           # it moved


def rot90(q, ny):
    """The state rotated by +90 degrees about the polar axis, as a
    permutation of cells: upper block cell (iu, j) -> (ny - 1 - j, iu), lower
    block cell (il, j) -> (j, ny - 1 - il); momenta (mx, my, mz) ->
    (-my, mx, mz)."""
    out = torch.empty_like(q)
    for j in range(ny):
        for i in range(ny):
            out[..., i, ny + ny - 1 - j] = q[..., j, ny + i]       # upper: new (ny-1-j, i) <- old (i, j)
            out[..., ny - 1 - i, j] = q[..., j, i]                 # lower: new (j, ny-1-i) <- old (i, j)
    m = out[:, 1:3].clone()
    out[:, 1] = -m[:, 1]
    out[:, 2] = m[:, 0]
    return out


@pytest.mark.parametrize("flux", FLUXES)
def test_rotation_equivariance(flux):
    """Rotating the initial state by 90 degrees about the polar axis rotates
    the solution: the mapping, both seams and the edge frames must all
    respect the grid's symmetry (a wrongly oriented normal in one sector or
    a seam glued without reversing its columns breaks it; the Coriolis term
    commutes with the rotation and is pinned by the inertial oscillation)."""
    ny = 8
    G = S.Grid(2 * ny, ny)
    q0 = bump_state(G, 2, vel=0.2)
    qa, _, dts = S.run(q0, G, 12, g=G_ND, omega=OMEGA, flux=flux)
    qb, _, _ = S.run(rot90(q0, ny), G, 12, g=G_ND, omega=OMEGA, dt_mode="replay", dts=dts[:, 0], flux=flux)
    scale = q0.abs().amax(dim=(0, 2, 3)).view(1, 4, 1, 1)
    assert float(((rot90(qa, ny) - qb).abs() / scale).max()) < 1e-12
    assert float(((qa - q0).abs() / scale).max()) > 1e-3


def coarsen(q, G_fine, G_coarse):
    """Area-weighted 2 x 2 block means (the fine cells tile the coarse ones)."""
    B, C, ny, nx = q.shape
    w = (q * G_fine.area).reshape(B, C, ny // 2, 2, nx // 2, 2).sum(dim=(3, 5))
    return w / G_coarse.area


def test_converges_on_a_smooth_flow():
    """Self-convergence on a smooth rotating flow at a fixed time: the change
    between successive refinements shrinks at better than first order."""
    grids = [S.Grid(2 * n, n) for n in (12, 24, 48)]
    out = []
    T = 0.02
    for G in grids:
        q0 = bump_state(G, 3, vel=0.3)
        dt = 0.4 / (48 * 40)
        steps = int(round(T / dt))
        q, _, _ = S.run(q0, G, steps, g=G_ND, omega=OMEGA, dt_mode="fixed", dt_fixed=T / steps)
        out.append(q)
    d1 = (out[0] - coarsen(out[1], grids[1], grids[0]))[:, 0].abs().mean()
    d2 = (out[1] - coarsen(out[2], grids[2], grids[1]))[:, 0].abs().mean()
    assert float(d1 / d2) > 2.5, (float(d1), float(d2))


def test_inertial_oscillation():
    """With a negligible pressure force (tiny g) and a tiny momentum (no
    advection), each cell's momentum turns about the local vertical at the
    inertial rate -2 Omega z (clockwise where z > 0): Eq. 3.2's Coriolis term
    in sign and magnitude, integrated by SSP-RK2."""
    G = S.Grid(24, 12)
    x = G.centre
    eps = 1e-9
    m0 = torch.cross(torch.tensor([0.3, -0.5, 0.8], dtype=torch.float64).expand_as(x), x, dim=-1) * eps
    q0 = torch.zeros(1, 4, 12, 24, dtype=torch.float64)
    q0[:, 0] = 1.0
    q0[0, 1:] = m0.permute(2, 0, 1)
    omega, T, steps = 1.0, 0.5, 200
    q, _, _ = S.run(q0, G, steps, g=1e-12, omega=omega, dt_mode="fixed", dt_fixed=T / steps)
    m = q[0, 1:].permute(1, 2, 0)
    z = x[..., 2]
    ang = torch.atan2((torch.cross(m0, m, dim=-1) * x).sum(-1), (m0 * m).sum(-1))
    sel = m0.norm(dim=-1) > 0.2 * eps
    want = -2.0 * omega * z * T
    assert float((ang - want)[sel].abs().max()) < 1e-5, float((ang - want)[sel].abs().max())
    assert float((m.norm(dim=-1) / m0.norm(dim=-1) - 1)[sel].abs().max()) < 1e-5
