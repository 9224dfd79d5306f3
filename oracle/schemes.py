"""FP64 oracle of the other numerical fluxes and the SSP-RK3 integrator
(test infrastructure only).

Section 2.3.3 lists, besides HLL (Eq. 2.15, in ``oracle.fv``):
  * Lax-Friedrichs (Eq. 2.11),
  * Rusanov (Eq. 2.12),
  * Roe (Eqs. 2.13, 2.14),
  * HLLE (Eq. 2.16),
  * HLLC (Eq. 2.17),
and Section 2.3.4 the three-stage TVD Runge-Kutta scheme of Eq. 2.20.  Each
flux here acts on two states already rotated into the face frame (component
1 = normal momentum), like ``oracle.fv.hll``; ``face_flux`` rotates, solves
and rotates back (Eq. 2.24).

Readings of the paper where it is garbled or silent (each one is listed with
its reason in the design notes):
  * Lax-Friedrichs: Eq. 2.11 is one-dimensional, with numerical viscosity
    dx / (2 dt).  In the unsplit 2D update that viscosity in both directions
    amplifies the grid-scale checkerboard mode by -3 for every dt, so each
    direction takes half of it, dx / (4 dt) on x faces and dy / (4 dt) on y
    faces (the first-order scheme is then the average of the four
    neighbours, the 2D Lax-Friedrichs scheme).
  * Rusanov: the printed s_R = max(|F'(Q_i)|, |F'(Q_{i+1})|) / 2 with
    |F'| the spectral radius |u_n| + c of each state.
  * Roe: Roe-averaged states (square-root-of-density weights; SWE depth the
    arithmetic mean), eigen-decomposition of the averaged Jacobian, no
    entropy fix (the paper states none).
  * HLLE: lambda_L = u_L - c_L, lambda_R = u_R + c_R, lambda_m the Roe
    state's u - c (for s_L) and u + c (for s_R), clamped by 0 as printed.
  * HLLC: the paper leaves the middle wave speed open; s_* from the jump
    conditions across the outer waves (Toro), outer speeds as for HLL (the
    Davis estimates), tangential momentum carried by the contact.
  * Eq. 2.20 is labelled "fourth order" but is the three-stage SSP-RK3 of
    Shu and Osher (third order).
"""
from __future__ import annotations

import torch

from . import fv

HLL = "hll"
RUSANOV = "rusanov"
LAX_FRIEDRICHS = "lf"
ROE = "roe"
HLLE = "hlle"
HLLC = "hllc"
FLUXES = (HLL, RUSANOV, LAX_FRIEDRICHS, ROE, HLLE, HLLC)

RK2 = 2
RK3 = 3


def _states(qL, qR, eq, g, gamma):
    uL, cL = fv.normal_velocity_and_sound_speed(qL, eq, g, gamma)
    uR, cR = fv.normal_velocity_and_sound_speed(qR, eq, g, gamma)
    FL = fv.normal_flux(qL, eq, g, gamma)
    FR = fv.normal_flux(qR, eq, g, gamma)
    return uL, cL, uR, cR, FL, FR


# ----------------------------------------------------------------------------
# Eq. 2.11 and Eq. 2.12: central fluxes with numerical viscosity
# ----------------------------------------------------------------------------

def lax_friedrichs(qL, qR, eq, g, gamma, nu):
    """1/2 (F_L + F_R) - nu (Q_R - Q_L) with the viscosity nu = d / (4 dt)
    of the face's direction (see the reading above)."""
    FL = fv.normal_flux(qL, eq, g, gamma)
    FR = fv.normal_flux(qR, eq, g, gamma)
    nu = torch.as_tensor(nu, dtype=qL.dtype)
    if nu.dim() > 0:
        nu = nu.view(-1, *([1] * (qL.dim() - 1)))
    return 0.5 * (FL + FR) - nu * (qR - qL)


def rusanov(qL, qR, eq, g, gamma):
    """1/2 (F_L + F_R) - s (Q_R - Q_L), s = max(|u_L| + c_L, |u_R| + c_R) / 2."""
    uL, cL, uR, cR, FL, FR = _states(qL, qR, eq, g, gamma)
    s = 0.5 * torch.maximum(uL.abs() + cL, uR.abs() + cR).unsqueeze(1)
    return 0.5 * (FL + FR) - s * (qR - qL)


# ----------------------------------------------------------------------------
# Eqs. 2.13 / 2.14: Roe
# ----------------------------------------------------------------------------

def roe_average(qL, qR, eq, g, gamma):
    """Roe state (u, v, c) and, for Euler, the enthalpy H, of two face-frame
    states."""
    rL, rR = qL[:, 0], qR[:, 0]
    sL, sR = torch.sqrt(rL), torch.sqrt(rR)
    u = (qL[:, 1] / sL + qR[:, 1] / sR) / (sL + sR)
    v = (qL[:, 2] / sL + qR[:, 2] / sR) / (sL + sR)
    if eq == fv.SWE:
        c = torch.sqrt(g * 0.5 * (rL + rR))
        return u, v, c, None
    pL, pR = fv.pressure(qL, gamma), fv.pressure(qR, gamma)
    HL, HR = (qL[:, 3] + pL) / rL, (qR[:, 3] + pR) / rR
    H = (sL * HL + sR * HR) / (sL + sR)
    c = torch.sqrt((gamma - 1.0) * (H - 0.5 * (u * u + v * v)))
    return u, v, c, H


def roe(qL, qR, eq, g, gamma):
    """1/2 (F_L + F_R) - 1/2 sum_p |lambda_p| alpha_p r_p on the Roe-averaged
    Jacobian (eigenvalues u - c, u (twice for Euler), u + c)."""
    FL = fv.normal_flux(qL, eq, g, gamma)
    FR = fv.normal_flux(qR, eq, g, gamma)
    u, v, c, H = roe_average(qL, qR, eq, g, gamma)
    d = qR - qL
    one, zero = torch.ones_like(u), torch.zeros_like(u)
    if eq == fv.SWE:
        a1 = ((u + c) * d[:, 0] - d[:, 1]) / (2 * c)
        a3 = (d[:, 1] - (u - c) * d[:, 0]) / (2 * c)
        a2 = d[:, 2] - v * d[:, 0]
        waves = [
            ((u - c).abs(), a1, torch.stack([one, u - c, v], dim=1)),
            (u.abs(), a2, torch.stack([zero, zero, one], dim=1)),
            ((u + c).abs(), a3, torch.stack([one, u + c, v], dim=1)),
        ]
    else:
        a3 = d[:, 2] - v * d[:, 0]
        dE = d[:, 3] - a3 * v
        a2 = (gamma - 1.0) / (c * c) * (d[:, 0] * (H - u * u) + u * d[:, 1] - dE)
        a1 = (d[:, 0] * (u + c) - d[:, 1] - c * a2) / (2 * c)
        a4 = d[:, 0] - (a1 + a2)
        waves = [
            ((u - c).abs(), a1, torch.stack([one, u - c, v, H - u * c], dim=1)),
            (u.abs(), a2, torch.stack([one, u, v, 0.5 * (u * u + v * v)], dim=1)),
            (u.abs(), a3, torch.stack([zero, zero, one, v], dim=1)),
            ((u + c).abs(), a4, torch.stack([one, u + c, v, H + u * c], dim=1)),
        ]
    diss = sum(lam.unsqueeze(1) * a.unsqueeze(1) * r for lam, a, r in waves)
    return 0.5 * (FL + FR) - 0.5 * diss


# ----------------------------------------------------------------------------
# Eq. 2.16: HLLE; Eq. 2.17: HLLC
# ----------------------------------------------------------------------------

def _hll_formula(qL, qR, FL, FR, sL, sR):
    F_hll = (sR * FL - sL * FR + sL * sR * (qR - qL)) / (sR - sL)
    return torch.where(sL >= 0, FL, torch.where(sR < 0, FR, F_hll))


def hlle(qL, qR, eq, g, gamma):
    """The HLL formula with s_L = min(u_L - c_L, u~ - c~, 0) and
    s_R = max(u_R + c_R, u~ + c~, 0), u~, c~ of the Roe state."""
    uL, cL, uR, cR, FL, FR = _states(qL, qR, eq, g, gamma)
    u, _, c, _ = roe_average(qL, qR, eq, g, gamma)
    zero = torch.zeros_like(u)
    sL = torch.minimum(torch.minimum(uL - cL, u - c), zero).unsqueeze(1)
    sR = torch.maximum(torch.maximum(uR + cR, u + c), zero).unsqueeze(1)
    return _hll_formula(qL, qR, FL, FR, sL, sR)


def _star_state(q, u_k, s_k, s_star, eq, gamma):
    """Q_*K = rho_K (s_K - u_K) / (s_K - s_*) [1, s_*, v_K, E_*] (Euler) or
    h_K (s_K - u_K) / (s_K - s_*) [1, s_*, v_K] (SWE)."""
    r = q[:, 0]
    fac = r * (s_k - u_k) / (s_k - s_star)
    v = q[:, 2] / r
    if eq == fv.SWE:
        return torch.stack([fac, fac * s_star, fac * v], dim=1)
    p = fv.pressure(q, gamma)
    e = q[:, 3] / r + (s_star - u_k) * (s_star + p / (r * (s_k - u_k)))
    return torch.stack([fac, fac * s_star, fac * v, fac * e], dim=1)


def hllc(qL, qR, eq, g, gamma):
    """F_L if 0 <= s_L; F_L + s_L (Q_*L - Q_L) if s_L <= 0 <= s_*;
    F_R + s_R (Q_*R - Q_R) if s_* <= 0 <= s_R; F_R if s_R <= 0."""
    uL, cL, uR, cR, FL, FR = _states(qL, qR, eq, g, gamma)
    sL = torch.minimum(uL - cL, uR - cR)
    sR = torch.maximum(uL + cL, uR + cR)
    rL, rR = qL[:, 0], qR[:, 0]
    if eq == fv.SWE:
        num = sL * rR * (uR - sR) - sR * rL * (uL - sL)
        den = rR * (uR - sR) - rL * (uL - sL)
    else:
        pL, pR = fv.pressure(qL, gamma), fv.pressure(qR, gamma)
        num = pR - pL + rL * uL * (sL - uL) - rR * uR * (sR - uR)
        den = rL * (sL - uL) - rR * (sR - uR)
    s_star = num / den
    FsL = FL + sL.unsqueeze(1) * (_star_state(qL, uL, sL, s_star, eq, gamma) - qL)
    FsR = FR + sR.unsqueeze(1) * (_star_state(qR, uR, sR, s_star, eq, gamma) - qR)
    sL_, sR_, ss = sL.unsqueeze(1), sR.unsqueeze(1), s_star.unsqueeze(1)
    return torch.where(sL_ >= 0, FL, torch.where(ss >= 0, FsL, torch.where(sR_ > 0, FsR, FR)))


def normal_flux_solver(name, qL, qR, eq, g, gamma, nu=None):
    if name == HLL:
        return fv.hll(qL, qR, eq, g, gamma)
    if name == RUSANOV:
        return rusanov(qL, qR, eq, g, gamma)
    if name == LAX_FRIEDRICHS:
        return lax_friedrichs(qL, qR, eq, g, gamma, nu)
    if name == ROE:
        return roe(qL, qR, eq, g, gamma)
    if name == HLLE:
        return hlle(qL, qR, eq, g, gamma)
    if name == HLLC:
        return hllc(qL, qR, eq, g, gamma)
    raise ValueError(name)


def face_flux(name, qL, qR, n, t, eq, g, gamma, nu=None):
    """Rotate into the face frame, solve, rotate back (Eq. 2.24)."""
    f = normal_flux_solver(name, fv.rotate(qL, n, t), fv.rotate(qR, n, t), eq, g, gamma, nu)
    return fv.rotate_back(f, n, t)


# ----------------------------------------------------------------------------
# Right-hand side and time integration
# ----------------------------------------------------------------------------

def rhs(q, eq, dx, dy, flux=HLL, dt=None, g=9.81, gamma=1.4, recon=None):
    """L(q) with MUSCL-minmod faces (or ``recon``) and the named flux; the
    Lax-Friedrichs flux needs the step's dt (per member)."""
    recon = recon or fv.muscl_minmod
    nu_x = nu_y = None
    if flux == LAX_FRIEDRICHS:
        dt = torch.as_tensor(dt, dtype=torch.float64).reshape(-1)
        nu_x, nu_y = dx / (4.0 * dt), dy / (4.0 * dt)
    QLx, QRx = recon(q, -1, dx)
    F = face_flux(flux, QLx, QRx, *fv.X_FACE, eq, g, gamma, nu_x)
    QLy, QRy = recon(q, -2, dy)
    G = face_flux(flux, QLy, QRy, *fv.Y_FACE, eq, g, gamma, nu_y)
    return fv.divergence_update(F, G, dx, dy)


def ssp_rk3(q, dt, L):
    """Eq. 2.20: q1 = q + dt L(q); q2 = 3/4 q + 1/4 q1 + 1/4 dt L(q1);
    q' = 1/3 q + 2/3 q2 + 2/3 dt L(q2)."""
    q1 = q + dt * L(q)
    q2 = 0.75 * q + 0.25 * q1 + 0.25 * dt * L(q1)
    return q / 3.0 + (2.0 / 3.0) * q2 + (2.0 / 3.0) * dt * L(q2)


def run(q0, eq, nsteps, *, flux=HLL, rk=RK2, cfl=0.5, dt_mode=fv.DT_ADAPTIVE, dt_fixed=None,
        dts=None, g=9.81, gamma=1.4, lx=1.0, ly=1.0, recon=None):
    """Like ``oracle.fv.run`` with a choice of flux and of SSP-RK2 / SSP-RK3;
    the adaptive dt is the same CFL rule (Eq. 2.10, 2D Courant number).
    Returns ``(q, t, dt_history[nsteps][B])``."""
    q = torch.as_tensor(q0, dtype=torch.float64).clone()
    B = q.shape[0]
    dx, dy = fv.grid_spacing(q, lx, ly)
    t = torch.zeros(B, dtype=torch.float64)
    hist = []
    for n in range(nsteps):
        if dt_mode == fv.DT_ADAPTIVE:
            dt = fv.cfl_dt(q, eq, cfl, dx, dy, g, gamma)
        elif dt_mode == fv.DT_FIXED:
            dt = torch.full((B,), float(dt_fixed), dtype=torch.float64)
        else:
            d = torch.as_tensor(dts[n], dtype=torch.float64)
            dt = d.expand(B).clone() if d.dim() == 0 else d.clone()

        def L(s, dt=dt):
            return rhs(s, eq, dx, dy, flux, dt, g, gamma, recon)

        step = fv.ssp_rk2 if rk == RK2 else ssp_rk3
        q = step(q, dt.view(B, 1, 1, 1), L)
        t = t + dt
        hist.append(dt)
    dt_hist = torch.stack(hist) if hist else torch.zeros(0, B, dtype=torch.float64)
    return q, t, dt_hist
