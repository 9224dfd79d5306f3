"""Pins of the oracle's other fluxes (Lax-Friedrichs, Rusanov, Roe, HLLE,
HLLC: Eqs. 2.11-2.17) and of SSP-RK3 (Eq. 2.20) against what the mathematics
fixes: consistency, exact upwinding, the Roe property (exact capture of a
stationary shock), exact resolution of contacts by Roe and HLLC, positivity
of HLLE in a strong rarefaction, the stability of the 2D Lax-Friedrichs
reading, the RK stability polynomials, and convergence to exact Riemann
solutions.  CPU only."""
import math

import numpy as np
import pytest
import torch

from oracle import fv, riemann
from oracle import schemes as S
from paper_2602_08670_gb300 import workloads as W

G = 9.81
GAMMA = 1.4
UPWIND = (S.HLL, S.ROE, S.HLLE, S.HLLC)


def swe(h, u, v):
    h, u, v = (torch.as_tensor(x, dtype=torch.float64).reshape(-1) for x in (h, u, v))
    return torch.stack([h, h * u, h * v], dim=1)


def euler(rho, u, v, p):
    rho, u, v, p = (torch.as_tensor(x, dtype=torch.float64).reshape(-1) for x in (rho, u, v, p))
    E = p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)
    return torch.stack([rho, rho * u, rho * v, E], dim=1)


def solve(name, qL, qR, eq, nu=1.0):
    return S.normal_flux_solver(name, qL, qR, eq, G, GAMMA, nu)


def random_states(eq, n=64, seed=0):
    g = torch.Generator().manual_seed(seed)
    r = lambda lo, hi: lo + (hi - lo) * torch.rand(n, generator=g, dtype=torch.float64)
    if eq == fv.SWE:
        return swe(r(0.5, 2.0), r(-1, 1), r(-1, 1)), swe(r(0.5, 2.0), r(-1, 1), r(-1, 1))
    return euler(r(0.3, 2), r(-1, 1), r(-1, 1), r(0.3, 2)), euler(r(0.3, 2), r(-1, 1), r(-1, 1), r(0.3, 2))


@pytest.mark.parametrize("eq", [fv.SWE, fv.EULER])
@pytest.mark.parametrize("name", S.FLUXES)
def test_consistency(name, eq):
    q, _ = random_states(eq)
    F = fv.normal_flux(q, eq, G, GAMMA)
    assert torch.allclose(solve(name, q, q, eq, nu=3.7), F, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("eq", [fv.SWE, fv.EULER])
@pytest.mark.parametrize("name", UPWIND)
def test_supersonic_states_take_the_left_flux(name, eq):
    """All waves moving right: the upwind fluxes return F_L.  For Roe this is
    the conservation property sum_p lambda_p alpha_p r_p = F_R - F_L of the
    Roe matrix, so it also pins the eigen-decomposition."""
    if eq == fv.SWE:
        qL, qR = swe([1.0, 0.8], [4.0, 5.0], [0.3, -0.2]), swe([1.2, 0.7], [4.5, 4.2], [0.1, 0.5])
    else:
        qL, qR = euler([1.0, 0.5], [2.0, 3.0], [0.2, -0.1], [0.5, 0.4]), euler([0.8, 0.6], [2.4, 2.9], [0.0, 0.3], [0.6, 0.3])
    out = solve(name, qL, qR, eq)
    assert torch.allclose(out, fv.normal_flux(qL, eq, G, GAMMA), rtol=1e-12, atol=1e-12)


def test_roe_captures_stationary_hydraulic_jump_exactly():
    """Conjugate depths of a standing hydraulic jump (Froude number 2.5):
    the jump satisfies the Rankine-Hugoniot conditions with speed 0, so the
    Roe flux equals F(q_L) = F(q_R); HLL smears it."""
    hL, uL = 1.0, 2.5 * math.sqrt(G)
    Fr = uL / math.sqrt(G * hL)
    hR = 0.5 * hL * (math.sqrt(1 + 8 * Fr * Fr) - 1)
    uR = hL * uL / hR
    qL, qR = swe(hL, uL, 0.2), swe(hR, uR, 0.2)
    FL, FR = fv.normal_flux(qL, fv.SWE, G, GAMMA), fv.normal_flux(qR, fv.SWE, G, GAMMA)
    assert torch.allclose(FL, FR, rtol=1e-13)
    out = solve(S.ROE, qL, qR, fv.SWE)
    assert torch.allclose(out, FL, rtol=1e-12, atol=1e-12)
    assert not torch.allclose(solve(S.HLL, qL, qR, fv.SWE)[:, :2], FL[:, :2], rtol=1e-3)


def test_roe_captures_stationary_normal_shock_exactly():
    """Normal shock at Mach 2 from the Rankine-Hugoniot relations (shock
    frame): the Roe flux equals F(q_L)."""
    M, rL, pL = 2.0, 1.0, 1.0
    cL = math.sqrt(GAMMA * pL / rL)
    uL = M * cL
    g = GAMMA
    rR = rL * (g + 1) * M * M / ((g - 1) * M * M + 2)
    pR = pL * (2 * g * M * M - (g - 1)) / (g + 1)
    uR = rL * uL / rR
    qL, qR = euler(rL, uL, 0.0, pL), euler(rR, uR, 0.0, pR)
    FL = fv.normal_flux(qL, fv.EULER, G, GAMMA)
    assert torch.allclose(FL, fv.normal_flux(qR, fv.EULER, G, GAMMA), rtol=1e-12)
    assert torch.allclose(solve(S.ROE, qL, qR, fv.EULER), FL, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("name", [S.ROE, S.HLLC])
def test_stationary_contact_and_shear_are_exact(name):
    """Density and tangential-velocity jump at rest with equal pressure: Roe
    and HLLC give the pressure flux (0, p, 0, 0) exactly (no mass diffused);
    HLL, HLLE and Rusanov diffuse it."""
    qL, qR = euler(1.0, 0.0, 0.3, 0.7), euler(0.25, 0.0, -0.4, 0.7)
    ref = torch.tensor([[0.0, 0.7, 0.0, 0.0]], dtype=torch.float64)
    assert torch.allclose(solve(name, qL, qR, fv.EULER), ref, atol=1e-14)
    for other in (S.HLL, S.HLLE, S.RUSANOV):
        assert abs(float(solve(other, qL, qR, fv.EULER)[0, 0])) > 1e-3


def test_hllc_swe_shear_layer_is_exact():
    qL, qR = swe(1.3, 0.0, 0.5), swe(1.3, 0.0, -0.8)
    ref = torch.tensor([[0.0, 0.5 * G * 1.3 * 1.3, 0.0]], dtype=torch.float64)
    assert torch.allclose(solve(S.HLLC, qL, qR, fv.SWE), ref, atol=1e-13)
    assert abs(float(solve(S.HLL, qL, qR, fv.SWE)[0, 2])) > 1e-3


def test_rusanov_is_lax_friedrichs_with_the_local_speed():
    qL, qR = random_states(fv.SWE, seed=3)
    uL, cL = fv.normal_velocity_and_sound_speed(qL, fv.SWE, G, GAMMA)
    uR, cR = fv.normal_velocity_and_sound_speed(qR, fv.SWE, G, GAMMA)
    nu = 0.5 * torch.maximum(uL.abs() + cL, uR.abs() + cR)
    a = solve(S.RUSANOV, qL, qR, fv.SWE)
    b = S.lax_friedrichs(qL, qR, fv.SWE, G, GAMMA, nu)
    assert torch.allclose(a, b, rtol=1e-14, atol=1e-14)


def test_hlle_keeps_the_strong_rarefaction_wet():
    """Two streams leaving each other at speed 5 (SWE): the HLLE intermediate
    state h_* = (s_R h_R - s_L h_L - (F_R - F_L)_h) / (s_R - s_L) stays
    positive (the solver is positivity preserving)."""
    qL, qR = swe(1.0, -5.0, 0.0), swe(1.0, 5.0, 0.0)
    uL, cL = fv.normal_velocity_and_sound_speed(qL, fv.SWE, G, GAMMA)
    uR, cR = fv.normal_velocity_and_sound_speed(qR, fv.SWE, G, GAMMA)
    u, _, c, _ = S.roe_average(qL, qR, fv.SWE, G, GAMMA)
    sL = torch.minimum(torch.minimum(uL - cL, u - c), torch.zeros(1, dtype=torch.float64))
    sR = torch.maximum(torch.maximum(uR + cR, u + c), torch.zeros(1, dtype=torch.float64))
    FL, FR = fv.normal_flux(qL, fv.SWE, G, GAMMA), fv.normal_flux(qR, fv.SWE, G, GAMMA)
    hstar = (sR * qR[:, 0] - sL * qL[:, 0] - (FR[:, 0] - FL[:, 0])) / (sR - sL)
    assert float(hstar) > 0
    F = solve(S.HLLE, qL, qR, fv.SWE)
    assert float(F[0, 0]) == pytest.approx(0.0, abs=1e-12)   # symmetric: no net mass flux


def test_lax_friedrichs_2d_reading_is_stable_on_the_checkerboard():
    """First-order faces, constant state plus a checkerboard of amplitude 1e-6:
    with the viscosity d/(4 dt) per direction one forward-Euler step maps the
    checkerboard to -1 times itself (the 2D Lax-Friedrichs average); the
    one-dimensional d/(2 dt) in both directions would map it to -3 times."""
    n = 16
    q = torch.zeros(1, 3, n, n, dtype=torch.float64)
    q[:, 0] = 1.0
    cb = torch.tensor([[(-1.0) ** (i + j) for i in range(n)] for j in range(n)], dtype=torch.float64)
    q[:, 0] += 1e-6 * cb
    dx = dy = 1.0 / n
    dt = 1e-3
    first = lambda Q, d, delta: fv.first_order_faces(Q, d)
    q1 = q + dt * S.rhs(q, fv.SWE, dx, dy, S.LAX_FRIEDRICHS, dt, recon=first)
    amp = float(((q1[0, 0] - 1.0) * cb).mean()) / 1e-6
    assert amp == pytest.approx(-1.0, abs=1e-6)


@pytest.mark.parametrize("rk", [S.RK2, S.RK3])
def test_rk_stability_polynomial(rk):
    """On dq/dt = lambda q the schemes reproduce the Taylor polynomial of
    exp(z) to the order of the method (z = lambda dt)."""
    lam, dt = -1.7, 0.3
    q = torch.ones(1, 1, 1, 1, dtype=torch.float64)
    L = lambda s: lam * s
    z = lam * dt
    out = (fv.ssp_rk2 if rk == S.RK2 else S.ssp_rk3)(q, dt, L)
    poly = 1 + z + z * z / 2 + (z ** 3 / 6 if rk == S.RK3 else 0.0)
    assert float(out) == pytest.approx(poly, rel=1e-14)


def _l1(a, b):
    return float((torch.as_tensor(a) - torch.as_tensor(b)).abs().mean())


def _run_to(q0, eq, T, flux, rk, cfl=0.45):
    q = torch.as_tensor(q0, dtype=torch.float64)
    dx, dy = fv.grid_spacing(q)
    t = 0.0
    while t < T - 1e-14:
        dt = min(float(fv.cfl_dt(q, eq, cfl, dx, dy).min()), T - t)
        q, _, _ = S.run(q, eq, 1, flux=flux, rk=rk, dt_mode=fv.DT_FIXED, dt_fixed=dt)
        t += dt
    return q


@pytest.mark.parametrize("flux,rk", [(S.RUSANOV, S.RK2), (S.LAX_FRIEDRICHS, S.RK2), (S.ROE, S.RK2),
                                     (S.HLLE, S.RK2), (S.HLLC, S.RK2), (S.HLL, S.RK3)])
def test_dam_break_converges_with_every_scheme(flux, rk):
    errs = []
    for n in (64, 256):
        q = _run_to(W.swe_dam_break(n, 2), fv.SWE, 0.06, flux, rk)
        ex = riemann.swe_dam_break_exact(n, 0.06)
        errs.append(_l1(q[0, 0, 0], ex[0]) + _l1(q[0, 1, 0], ex[1]))
        assert float(q[0, 2].abs().max()) == 0.0
    rate = math.log2(errs[0] / errs[1]) / 2
    assert rate > 0.6 and errs[1] < 3e-2, (errs, rate)


@pytest.mark.parametrize("flux", [S.ROE, S.HLLC])
def test_sod_converges_with_contact_resolving_fluxes(flux):
    errs = []
    for n in (64, 256):
        q = _run_to(W.euler_sod(n, 2, axis="x"), fv.EULER, 0.1, flux, S.RK2)
        ex = riemann.euler_sod_exact(n, 0.1)
        errs.append(_l1(q[0, 0, 0], ex[0]) + _l1(q[0, 1, 0], ex[1]) + _l1(q[0, 3, 0], ex[2]))
    rate = math.log2(errs[0] / errs[1]) / 2
    assert rate > 0.6 and errs[1] < 3e-2, (errs, rate)


def test_rk3_linear_wave_second_order_in_space():
    errs = []
    for n in (32, 128):
        q = _run_to(W.swe_linear_wave(n, 2), fv.SWE, 0.1, S.HLL, S.RK3)
        x = W.cell_centres(n)
        exact = 1.0 + 1e-6 * np.sin(2 * math.pi * (x - math.sqrt(G) * 0.1))
        errs.append(np.abs(q[0, 0, 0].numpy() - exact).mean())
    assert math.log2(errs[0] / errs[1]) / 2 > 1.7, errs
