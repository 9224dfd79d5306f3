"""Pins of the FP64 oracle of the plain step against what the mathematics and
the paper fix: exact Riemann solutions, linear-wave propagation, invariants
(lake at rest, conservation, translation and transpose symmetry), closed
forms of the flux, limiter and reconstruction.  CPU only."""
import math

import numpy as np
import pytest
import torch

from oracle import fv, riemann
from paper_2602_08670_gb300 import workloads as W

G = 9.81
GAMMA = 1.4


def run_to_time(q0, eq, T, cfl=0.45):
    """Advance to exactly time T (last step shortened)."""
    q = torch.as_tensor(q0, dtype=torch.float64)
    dx, dy = fv.grid_spacing(q)
    t = 0.0
    while t < T - 1e-14:
        dt = min(float(fv.cfl_dt(q, eq, cfl, dx, dy).min()), T - t)
        q, _, _, _ = fv.run(q, eq, 1, dt_mode=fv.DT_FIXED, dt_fixed=dt)
        t += dt
    return q


# --------------------------------------------------------------------------
# Eq. 2.18 limiter and reconstruction
# --------------------------------------------------------------------------

def test_minmod_table():
    a = torch.tensor([1.0, 3.0, -2.0, -0.5, 2.0, 0.0, 1.0, -4.0])
    b = torch.tensor([3.0, 1.0, -0.5, -2.0, -1.0, 5.0, 0.0, -4.0])
    expect = torch.tensor([1.0, 1.0, -0.5, -0.5, 0.0, 0.0, 0.0, -4.0])
    assert torch.equal(fv.minmod(a, b), expect)


def test_reconstruction_constant_exact():
    Q = torch.full((1, 3, 6, 8), 1.25, dtype=torch.float64)
    for dim, d in ((-1, 1 / 8), (-2, 1 / 6)):
        QL, QR = fv.muscl_minmod(Q, dim, d)
        assert torch.equal(QL, Q) and torch.equal(QR, Q)


def test_reconstruction_linear_exact_interior():
    # Q_i = a + s x_i with x_i the cell centre; the face value at x_{i+1/2}
    # is a + s (i+1) dx from both sides (this fixes the sign of Q^R).
    n = 16
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    Q = torch.zeros(1, 3, 1, n, dtype=torch.float64)
    Q[0, 0, 0] = torch.tensor(2.0 + 3.0 * x)
    Q[0, 1, 0] = torch.tensor(-1.0 + 0.5 * x)
    Q[0, 2, 0] = torch.tensor(0.25 - 2.0 * x)
    QL, QR = fv.muscl_minmod(Q, -1, dx)
    face = torch.tensor((np.arange(n) + 1) * dx)
    interior = slice(1, n - 2)   # faces whose stencil does not cross the wrap
    for c, (a, s) in enumerate(((2.0, 3.0), (-1.0, 0.5), (0.25, -2.0))):
        exact = a + s * face
        assert torch.allclose(QL[0, c, 0, interior], exact[interior], rtol=0, atol=1e-14)
        assert torch.allclose(QR[0, c, 0, interior], exact[interior], rtol=0, atol=1e-14)


def test_reconstruction_limits_at_extremum():
    # at a local maximum the slope is zero: both faces of that cell equal Q_i
    Q = torch.tensor([[[[1.0, 2.0, 5.0, 3.0, 1.0, 0.5]]]]).repeat(1, 3, 1, 1)
    QL, QR = fv.muscl_minmod(Q, -1, 1.0)
    assert float(QL[0, 0, 0, 2]) == 5.0          # Q^L_{2+1/2} = Q_2
    assert float(QR[0, 0, 0, 1]) == 5.0          # Q^R_{1+1/2} = Q_2


# --------------------------------------------------------------------------
# Eq. 2.15 HLL and Eq. 2.24 rotation
# --------------------------------------------------------------------------

def _swe_state(h, u, v):
    return torch.tensor([[h, h * u, h * v]], dtype=torch.float64)


def _euler_state(rho, u, v, p):
    return torch.tensor([[rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)]],
                        dtype=torch.float64)


def test_swe_physical_flux_closed_form():
    q = _swe_state(2.0, 0.3, -0.7)
    F = fv.normal_flux(q, fv.SWE, G, GAMMA)[0]
    expect = [2.0 * 0.3, 2.0 * 0.09 + 0.5 * G * 4.0, 2.0 * 0.3 * -0.7]
    assert np.allclose(F.numpy(), expect, rtol=1e-15, atol=1e-15)


def test_euler_physical_flux_closed_form():
    rho, u, v, p = 1.3, 0.4, -0.2, 2.1
    q = _euler_state(rho, u, v, p)
    E = float(q[0, 3])
    F = fv.normal_flux(q, fv.EULER, G, GAMMA)[0]
    expect = [rho * u, rho * u * u + p, rho * u * v, u * (E + p)]
    assert np.allclose(F.numpy(), expect, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("eq", [fv.SWE, fv.EULER])
def test_hll_consistency(eq):
    rng = np.random.default_rng(0)
    for _ in range(20):
        if eq == fv.SWE:
            q = _swe_state(rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1))
        else:
            q = _euler_state(rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1),
                             rng.uniform(0.5, 2))
        F = fv.hll(q, q, eq, G, GAMMA)
        assert torch.allclose(F, fv.normal_flux(q, eq, G, GAMMA), rtol=1e-14, atol=1e-14)


def test_hll_supersonic_upwinding_exact():
    qL = _swe_state(1.0, 5.0, 0.2)    # u - c > 0 on both sides: s_L > 0
    qR = _swe_state(1.1, 5.2, -0.1)
    assert torch.equal(fv.hll(qL, qR, fv.SWE, G, GAMMA), fv.normal_flux(qL, fv.SWE, G, GAMMA))
    qL = _swe_state(1.0, -5.0, 0.2)   # s_R < 0
    qR = _swe_state(1.1, -5.2, -0.1)
    assert torch.equal(fv.hll(qL, qR, fv.SWE, G, GAMMA), fv.normal_flux(qR, fv.SWE, G, GAMMA))


@pytest.mark.parametrize("hL,uL,hR,uR", [(1.0, 0.1, 0.6, -0.2), (0.6, 0.2, 1.0, -0.1),
                                          (0.8, -0.5, 1.4, 0.9), (1.5, 1.0, 0.7, 2.5)])
def test_hll_swe_closed_form(hL, uL, hR, uR):
    qL, qR = _swe_state(hL, uL, 0.3), _swe_state(hR, uR, -0.4)
    cL, cR = math.sqrt(G * hL), math.sqrt(G * hR)
    sL, sR = min(uL - cL, uR - cR), max(uL + cL, uR + cR)
    FL = np.array([hL * uL, hL * uL * uL + 0.5 * G * hL * hL, hL * uL * 0.3])
    FR = np.array([hR * uR, hR * uR * uR + 0.5 * G * hR * hR, hR * uR * -0.4])
    dq = qR[0].numpy() - qL[0].numpy()
    if sL >= 0:
        expect = FL
    elif sR < 0:
        expect = FR
    else:
        expect = (sR * FL - sL * FR + sL * sR * dq) / (sR - sL)
    assert np.allclose(fv.hll(qL, qR, fv.SWE, G, GAMMA)[0].numpy(), expect, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("L,R", [((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),
                                 ((0.125, 0.2, 0.1), (1.0, -0.3, 1.0)),
                                 ((1.2, 2.5, 0.4), (1.0, 2.0, 0.5))])
def test_hll_euler_closed_form(L, R):
    (rL, uL, pL), (rR, uR, pR) = L, R
    qL, qR = _euler_state(rL, uL, 0.1, pL), _euler_state(rR, uR, -0.2, pR)
    EL, ER = float(qL[0, 3]), float(qR[0, 3])
    cL, cR = math.sqrt(GAMMA * pL / rL), math.sqrt(GAMMA * pR / rR)
    sL, sR = min(uL - cL, uR - cR), max(uL + cL, uR + cR)
    FL = np.array([rL * uL, rL * uL * uL + pL, rL * uL * 0.1, uL * (EL + pL)])
    FR = np.array([rR * uR, rR * uR * uR + pR, rR * uR * -0.2, uR * (ER + pR)])
    dq = qR[0].numpy() - qL[0].numpy()
    if sL >= 0:
        expect = FL
    elif sR < 0:
        expect = FR
    else:
        expect = (sR * FL - sL * FR + sL * sR * dq) / (sR - sL)
    assert np.allclose(fv.hll(qL, qR, fv.EULER, G, GAMMA)[0].numpy(), expect, rtol=1e-13, atol=1e-14)


def test_rotation_y_face_equals_y_flux():
    # through a y-face the flux must be G(q) = (hv, hu v, hv^2/h + g h^2/2)
    q = _swe_state(1.7, 0.4, -0.9)
    Fy = fv.face_flux(q, q, *fv.Y_FACE, fv.SWE, G, GAMMA)[0].numpy()
    h, hu, hv = q[0].numpy()
    expect = [hv, hu * hv / h, hv * hv / h + 0.5 * G * h * h]
    assert np.allclose(Fy, expect, rtol=1e-14, atol=1e-14)


def test_rotation_is_orthogonal():
    q = torch.randn(5, 4, dtype=torch.float64)
    for n, t in (fv.X_FACE, fv.Y_FACE, ((0.6, 0.8), (-0.8, 0.6))):
        assert torch.allclose(fv.rotate_back(fv.rotate(q, n, t), n, t), q, atol=1e-15)


# --------------------------------------------------------------------------
# Invariants of the full step
# --------------------------------------------------------------------------

def test_lake_at_rest_bitwise():
    q0 = torch.zeros(1, 3, 12, 10, dtype=torch.float64)
    q0[:, 0] = 1.3
    q, _, _, _ = fv.run(q0, fv.SWE, 20)
    assert torch.equal(q, q0)


def test_uniform_euler_flow_bitwise():
    q0 = _euler_state(1.2, 0.3, -0.4, 0.9).view(1, 4, 1, 1).repeat(1, 1, 8, 12)
    q, _, _, _ = fv.run(q0, fv.EULER, 20)
    assert torch.equal(q, q0)


@pytest.mark.parametrize("eq", [fv.SWE, fv.EULER])
def test_conservation_to_roundoff(eq):
    if eq == fv.SWE:
        q0 = torch.tensor(W.random_smooth_swe(32, seed=3, vel=0.2))
    else:
        q0 = torch.tensor(W.euler_kelvin_helmholtz(32, 32, seed=1))
    d0 = fv.diagnostics(q0, eq)
    q, _, _, _ = fv.run(q0, eq, 200)
    d1 = fv.diagnostics(q, eq)
    C = q0.shape[1]
    scale = d0[0, :C].abs().max()
    assert float((d1[0, :C] - d0[0, :C]).abs().max() / scale) < 1e-13


def test_translation_invariance_bitwise():
    q0 = torch.tensor(W.random_smooth_swe(24, seed=5, vel=0.2))
    q, _, _, _ = fv.run(q0, fv.SWE, 10, dt_mode=fv.DT_FIXED, dt_fixed=1e-3)
    qs, _, _, _ = fv.run(torch.roll(q0, (5, 7), (-2, -1)), fv.SWE, 10,
                         dt_mode=fv.DT_FIXED, dt_fixed=1e-3)
    assert torch.equal(torch.roll(q, (5, 7), (-2, -1)), qs)


def test_transpose_symmetry_bitwise():
    q0 = torch.tensor(W.random_smooth_swe(16, seed=7, vel=0.2))
    qt = q0.transpose(-1, -2)[:, [0, 2, 1]].contiguous()
    q, _, _, _ = fv.run(q0, fv.SWE, 10, dt_mode=fv.DT_FIXED, dt_fixed=1e-3)
    qT, _, _, _ = fv.run(qt, fv.SWE, 10, dt_mode=fv.DT_FIXED, dt_fixed=1e-3)
    assert torch.equal(q.transpose(-1, -2)[:, [0, 2, 1]], qT)


def test_cfl_dt_closed_form():
    H, u, v = 2.0, 0.3, -0.5
    q = _swe_state(H, u, v).view(1, 3, 1, 1).repeat(1, 1, 4, 8)
    dt = float(fv.cfl_dt(q, fv.SWE, 0.5, 1 / 8, 1 / 4)[0])
    c = math.sqrt(G * H)
    assert dt == pytest.approx(0.5 / ((abs(u) + c) * 8 + (abs(v) + c) * 4), rel=1e-15)


def test_cfl_step_is_stable_to_grid_scale_noise():
    # At the adaptive dt the scheme must not amplify roundoff-size noise: a
    # 6e-8 relative perturbation of the bump workload stays below 1e-5 of the
    # solution after 100 steps (an unstable dt amplifies it by orders of
    # magnitude).
    q0 = torch.tensor(W.swe_gaussian_bump(64, 64))
    g = torch.Generator().manual_seed(0)
    qp = q0 * (1 + 6e-8 * torch.randn(q0.shape, generator=g, dtype=torch.float64))
    qa, _, dts, _ = fv.run(q0, fv.SWE, 100, cfl=0.5)
    qb, _, _, _ = fv.run(qp, fv.SWE, 100, dt_mode=fv.DT_REPLAY, dts=dts[:, 0])
    for c in range(3):
        rel = float((qa[:, c] - qb[:, c]).norm() / qa[:, c].norm())
        assert rel < 1e-5, (c, rel)


def test_batch_members_independent():
    a = torch.tensor(W.random_smooth_swe(16, seed=1, vel=0.1))
    b = torch.tensor(W.swe_gaussian_bump(16, 16))
    qa, ta, _, _ = fv.run(a, fv.SWE, 5)
    qb, tb, _, _ = fv.run(b, fv.SWE, 5)
    qab, tab, _, _ = fv.run(torch.cat([a, b]), fv.SWE, 5)
    assert torch.equal(qab, torch.cat([qa, qb])) and torch.equal(tab, torch.cat([ta, tb]))


def test_replay_equals_adaptive():
    q0 = torch.tensor(W.swe_gaussian_bump(32, 32))
    qa, _, dts, _ = fv.run(q0, fv.SWE, 8)
    qr, _, _, _ = fv.run(q0, fv.SWE, 8, dt_mode=fv.DT_REPLAY, dts=dts[:, 0])
    assert torch.equal(qa, qr)


# --------------------------------------------------------------------------
# Exact solutions
# --------------------------------------------------------------------------

def _l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).mean())


def test_swe_dam_break_converges_to_exact():
    errs = []
    for n in (64, 512):
        q = run_to_time(W.swe_dam_break(n, 2), fv.SWE, 0.06)
        ex = riemann.swe_dam_break_exact(n, 0.06)
        errs.append(_l1(q[0, 0, 0], ex[0]) + _l1(q[0, 1, 0], ex[1]))
        assert torch.equal(q[0, :, 0], q[0, :, 1])        # stays y-uniform
        assert float(q[0, 2].abs().max()) == 0.0          # no transverse momentum
    rate = math.log2(errs[0] / errs[1]) / 3
    assert rate > 0.8 and errs[1] < 1e-2, (errs, rate)


def test_swe_dam_break_star_state():
    # closed form check of the exact solver itself: the star state satisfies
    # the shock jump and the rarefaction invariant (h_L = 1, h_R = 0.35)
    hs, us = riemann.swe_star(1.0, 0.0, 0.35, 0.0, G)
    assert us == pytest.approx(2 * (math.sqrt(G) - math.sqrt(G * hs)), rel=1e-12)
    assert us == pytest.approx((hs - 0.35) * math.sqrt(0.5 * G * (hs + 0.35) / (hs * 0.35)), rel=1e-12)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_sod_converges_to_exact(axis):
    errs = []
    for n in (64, 512):
        nx, ny = (n, 2) if axis == "x" else (2, n)
        q0 = W.euler_sod(nx, ny, axis=axis)
        q = run_to_time(q0, fv.EULER, 0.1)
        ex = riemann.euler_sod_exact(n, 0.1)
        if axis == "x":
            rho, mom, E = q[0, 0, 0], q[0, 1, 0], q[0, 3, 0]
            assert float(q[0, 2].abs().max()) == 0.0
        else:
            rho, mom, E = q[0, 0, :, 0], q[0, 2, :, 0], q[0, 3, :, 0]
            assert float(q[0, 1].abs().max()) == 0.0
        errs.append(_l1(rho, ex[0]) + _l1(mom, ex[1]) + _l1(E, ex[2]))
    rate = math.log2(errs[0] / errs[1]) / 3
    assert rate > 0.8 and errs[1] < 1.5e-2, (errs, rate)


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_sod_star_state_textbook_values():
    """The exact Sod solution against the published star state (fixture
    tests/golden/sod_star_toro.txt): pressure and velocity of the star
    region, and the densities on either side of the contact sampled from the
    exact solution (left of it: the isentrope behind the rarefaction; right:
    the shock's Hugoniot)."""
    ref = _golden("sod_star_toro.txt")
    ps, us = riemann.euler_star(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, GAMMA)
    assert ps == pytest.approx(ref["p_star"], abs=1e-5)
    assert us == pytest.approx(ref["u_star"], abs=1e-5)
    xi = np.array([us - 1e-3, us + 1e-3])
    rho, u, p = riemann.euler_sample(xi, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, GAMMA)
    assert rho[0] == pytest.approx(ref["rho_star_left"], abs=1e-5)
    assert rho[1] == pytest.approx(ref["rho_star_right"], abs=1e-5)
    assert p[0] == pytest.approx(ref["p_star"], abs=1e-5) and p[1] == pytest.approx(ref["p_star"], abs=1e-5)


@pytest.mark.parametrize("eq", [fv.SWE, fv.EULER])
def test_linear_wave_second_order(eq):
    errs1, errsi = [], []
    for n in (32, 128):
        if eq == fv.SWE:
            q0, T, c = W.swe_linear_wave(n, 2), 0.1, math.sqrt(G)
        else:
            q0, T, c = W.euler_acoustic_wave(n, 2), 0.2, math.sqrt(GAMMA)
        q = run_to_time(q0, eq, T)
        x = W.cell_centres(n)
        exact = 1.0 + 1e-6 * np.sin(2 * math.pi * (x - c * T))
        d = q[0, 0, 0].numpy() - exact
        errs1.append(np.abs(d).mean())
        errsi.append(np.abs(d).max())
    r1 = math.log2(errs1[0] / errs1[1]) / 2
    ri = math.log2(errsi[0] / errsi[1]) / 2
    assert r1 > 1.7 and ri > 1.0, (r1, ri)


# --------------------------------------------------------------------------
# Diagnostics and coarse graining
# --------------------------------------------------------------------------

def test_energy_closed_form_at_rest():
    q = torch.zeros(1, 3, 8, 8, dtype=torch.float64)
    q[:, 0] = 1.5
    d = fv.diagnostics(q, fv.SWE)[0]
    assert float(d[0]) == pytest.approx(1.5, rel=1e-15)
    assert float(d[3]) == pytest.approx(0.5 * G * 1.5 ** 2, rel=1e-15)


def test_energy_moving_uniform():
    h, u, v = 2.0, 0.5, -1.0
    q = _swe_state(h, u, v).view(1, 3, 1, 1).repeat(1, 1, 4, 4)
    d = fv.diagnostics(q, fv.SWE)[0]
    assert float(d[3]) == pytest.approx(0.5 * G * h * h + 0.5 * (u * u + v * v) * h, rel=1e-14)


def test_coarsen_block_mean():
    q = torch.arange(2 * 3 * 8 * 8, dtype=torch.float64).reshape(2, 3, 8, 8)
    c = fv.coarsen(q, 4)
    assert c.shape == (2, 3, 2, 2)
    assert float(c[1, 2, 1, 0]) == float(q[1, 2, 4:8, 0:4].mean())
    assert torch.allclose(c.sum(dim=(2, 3)) * 16, q.sum(dim=(2, 3)))


def test_potential_enstrophy_closed_form():
    # Plane wave theta = 2 pi (x + 2 y) with u = -A sin(theta), v = B sin(theta)
    # on a constant depth H = 2.  Centred differences of sin(theta) are exact
    # multiples of cos(theta): d/dx -> s1 cos(theta), d/dy -> s2 cos(theta) with
    # s_k = n sin(2 pi k / n) / 1 (one and two wavelengths across the square).
    # So zeta = (B s1 + A s2) cos(theta) at every cell and, since cos^2 averages
    # to 1/2 over the grid, the integral of zeta^2 / (2 h) is
    # (B s1 + A s2)^2 / (4 H).  A swapped derivative axis gives B s2 + A s1, a
    # wrong sign B s1 - A s2, a missing 1/2 or 1/h a factor 2 or H.
    n, A, B, H = 32, 0.3, 0.7, 2.0
    X, Y = np.meshgrid(W.cell_centres(n), W.cell_centres(n))
    th = 2 * np.pi * (X + 2 * Y)
    q = torch.zeros(1, 3, n, n, dtype=torch.float64)
    q[0, 0] = H
    q[0, 1] = torch.tensor(H * (-A * np.sin(th)))
    q[0, 2] = torch.tensor(H * (B * np.sin(th)))
    s1 = n * np.sin(2 * np.pi / n)
    s2 = n * np.sin(4 * np.pi / n)
    expect = (B * s1 + A * s2) ** 2 / (4 * H)
    pe = float(fv.potential_enstrophy(q)[0])
    assert abs(pe - expect) <= 1e-12 * expect, (pe, expect)
    # u = v along the same wave: dv/dx = du/dy only when s1 = s2, so use the
    # diagonal wave theta = 2 pi (x + y), for which zeta vanishes identically
    th = 2 * np.pi * (X + Y)
    q[0, 1] = torch.tensor(H * 0.4 * np.sin(th))
    q[0, 2] = torch.tensor(H * 0.4 * np.sin(th))
    assert float(fv.potential_enstrophy(q)[0]) < 1e-24


def test_mean_relative_h_error_closed_forms():
    # Section 3's metric: mean over cells of |h_high - h_low| / h_high.
    # h_low = h_high (1 + eps_ij) with eps = +-e0 in a checkerboard gives
    # exactly e0 (a signed mean would give 0); h_low = 2 h_high gives 1 and
    # the swapped arguments 1/2 (the normalisation is by the high-resolution
    # depth).
    rng = np.random.default_rng(5)
    hh = torch.tensor(1.0 + rng.uniform(0.0, 0.5, size=(2, 16, 16)))
    sign = torch.tensor(np.where((np.add.outer(np.arange(16), np.arange(16)) % 2) == 0, 1.0, -1.0))
    e0 = 0.0625
    hl = hh * (1.0 + e0 * sign)
    assert abs(fv.mean_relative_h_error(hl, hh) - e0) < 1e-15
    assert fv.mean_relative_h_error(2 * hh, hh) == 1.0
    assert abs(fv.mean_relative_h_error(hh, 2 * hh) - 0.5) < 1e-15
    assert fv.mean_relative_h_error(hh, hh) == 0.0
