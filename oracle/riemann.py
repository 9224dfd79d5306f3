"""Exact Riemann solutions used to pin the oracle (test infrastructure only).

Two textbook problems with closed-form structure the thesis itself uses as
test cases: the shallow-water dam break (Section 3.1, initial h = 1 / 0.35)
and the Sod shock tube (Section 4.1, gamma = 7/5).  Both are solved exactly:
the star state from the scalar nonlinear equation of each system (root by
bracketing), then sampling of the self-similar solution at xi = x / t
(rarefaction fans from the Riemann invariants, shocks from the
Rankine-Hugoniot conditions).  The formulas are the standard ones of the
exact Riemann solvers in Toro, "Riemann Solvers and Numerical Methods for
Fluid Dynamics" (the thesis's reference for its HLL flux).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


# ----------------------------------------------------------------------------
# Shallow water, wet bed on both sides
# ----------------------------------------------------------------------------

def _swe_f(h, hk, g):
    """Velocity jump across the wave connecting depth hk to depth h."""
    if h <= hk:   # rarefaction: Riemann invariant u +- 2 sqrt(g h)
        return 2.0 * (math.sqrt(g * h) - math.sqrt(g * hk))
    return (h - hk) * math.sqrt(0.5 * g * (h + hk) / (h * hk))   # shock


def swe_star(hL, uL, hR, uR, g):
    fun = lambda h: _swe_f(h, hL, g) + _swe_f(h, hR, g) + uR - uL
    hs = brentq(fun, 1e-12, 10.0 * max(hL, hR) + 10.0, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (uL + uR) + 0.5 * (_swe_f(hs, hR, g) - _swe_f(hs, hL, g))
    return hs, us


def swe_sample(xi: np.ndarray, hL, uL, hR, uR, g):
    """Exact (h, u) of the shallow-water Riemann problem at xi = x / t."""
    hs, us = swe_star(hL, uL, hR, uR, g)
    aL, aR, a_s = math.sqrt(g * hL), math.sqrt(g * hR), math.sqrt(g * hs)
    h = np.empty_like(xi)
    u = np.empty_like(xi)
    for i, s in enumerate(xi):
        if s <= us:   # left of the contact (there is none for SWE; the star region)
            if hs > hL:   # left shock, speed from mass conservation
                S = (hs * us - hL * uL) / (hs - hL)
                h[i], u[i] = (hL, uL) if s < S else (hs, us)
            else:
                head, tail = uL - aL, us - a_s
                if s < head:
                    h[i], u[i] = hL, uL
                elif s > tail:
                    h[i], u[i] = hs, us
                else:
                    a = (uL + 2.0 * aL - s) / 3.0
                    h[i], u[i] = a * a / g, (uL + 2.0 * aL + 2.0 * s) / 3.0
        else:
            if hs > hR:
                S = (hs * us - hR * uR) / (hs - hR)
                h[i], u[i] = (hR, uR) if s > S else (hs, us)
            else:
                head, tail = uR + aR, us + a_s
                if s > head:
                    h[i], u[i] = hR, uR
                elif s < tail:
                    h[i], u[i] = hs, us
                else:
                    a = (-uR + 2.0 * aR + s) / 3.0
                    h[i], u[i] = a * a / g, (uR - 2.0 * aR + 2.0 * s) / 3.0
    return h, u


# ----------------------------------------------------------------------------
# Euler (ideal gas)
# ----------------------------------------------------------------------------

def _euler_f(p, rk, pk, gamma):
    ak = math.sqrt(gamma * pk / rk)
    if p > pk:   # shock
        A = 2.0 / ((gamma + 1.0) * rk)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * ak / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def euler_star(rL, uL, pL, rR, uR, pR, gamma):
    fun = lambda p: _euler_f(p, rL, pL, gamma) + _euler_f(p, rR, pR, gamma) + uR - uL
    ps = brentq(fun, 1e-14, 100.0 * max(pL, pR) + 10.0, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (uL + uR) + 0.5 * (_euler_f(ps, rR, pR, gamma) - _euler_f(ps, rL, pL, gamma))
    return ps, us


def euler_sample(xi: np.ndarray, rL, uL, pL, rR, uR, pR, gamma):
    """Exact (rho, u, p) of the Euler Riemann problem at xi = x / t."""
    ps, us = euler_star(rL, uL, pL, rR, uR, pR, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    aL, aR = math.sqrt(gamma * pL / rL), math.sqrt(gamma * pR / rR)
    out = np.empty((3, xi.size))
    for i, s in enumerate(xi):
        if s <= us:
            if ps > pL:
                rs = rL * (ps / pL + g1) / (g1 * ps / pL + 1.0)
                S = uL - aL * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pL
                                        + (gamma - 1.0) / (2 * gamma))
                out[:, i] = (rL, uL, pL) if s < S else (rs, us, ps)
            else:
                rs = rL * (ps / pL) ** (1.0 / gamma)
                a_s = aL * (ps / pL) ** ((gamma - 1.0) / (2 * gamma))
                if s < uL - aL:
                    out[:, i] = (rL, uL, pL)
                elif s > us - a_s:
                    out[:, i] = (rs, us, ps)
                else:
                    base = 2.0 / (gamma + 1.0) + (gamma - 1.0) / ((gamma + 1.0) * aL) * (uL - s)
                    out[:, i] = (rL * base ** (2.0 / (gamma - 1.0)),
                                 2.0 / (gamma + 1.0) * (aL + 0.5 * (gamma - 1.0) * uL + s),
                                 pL * base ** (2.0 * gamma / (gamma - 1.0)))
        else:
            if ps > pR:
                rs = rR * (ps / pR + g1) / (g1 * ps / pR + 1.0)
                S = uR + aR * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pR
                                        + (gamma - 1.0) / (2 * gamma))
                out[:, i] = (rR, uR, pR) if s > S else (rs, us, ps)
            else:
                rs = rR * (ps / pR) ** (1.0 / gamma)
                a_s = aR * (ps / pR) ** ((gamma - 1.0) / (2 * gamma))
                if s > uR + aR:
                    out[:, i] = (rR, uR, pR)
                elif s < us + a_s:
                    out[:, i] = (rs, us, ps)
                else:
                    base = 2.0 / (gamma + 1.0) - (gamma - 1.0) / ((gamma + 1.0) * aR) * (uR - s)
                    out[:, i] = (rR * base ** (2.0 / (gamma - 1.0)),
                                 2.0 / (gamma + 1.0) * (-aR + 0.5 * (gamma - 1.0) * uR + s),
                                 pR * base ** (2.0 * gamma / (gamma - 1.0)))
    return out


# ----------------------------------------------------------------------------
# Cell averages of the periodic two-problem solutions
# ----------------------------------------------------------------------------

def _periodic_xi(x: np.ndarray, t: float):
    """Map x in [0, 1) to (problem id, xi): problem 0 is centred at x = 1/2,
    problem 1 at x = 0 (= 1); each owns the half of the domain around it."""
    near_half = (x >= 0.25) & (x < 0.75)
    xi = np.where(near_half, (x - 0.5) / t, (np.mod(x + 0.5, 1.0) - 0.5) / t)
    return near_half, xi


def _cell_average(sampler, n: int, sub: int):
    xs = (np.arange(n * sub) + 0.5) / (n * sub)
    vals = sampler(xs)
    return vals.reshape(vals.shape[:-1] + (n, sub)).mean(axis=-1)


def swe_dam_break_exact(n: int, t: float, h_left=1.0, h_right=0.35, g=9.81, sub=16):
    """Cell averages of (h, hu) on n periodic cells for the workload
    ``swe_dam_break`` (jump at x = 1/2 and at x = 0), valid while the two
    problems' waves stay inside their halves."""
    def sampler(x):
        near, xi = _periodic_xi(x, t)
        h0, u0 = swe_sample(xi, h_left, 0.0, h_right, 0.0, g)
        h1, u1 = swe_sample(xi, h_right, 0.0, h_left, 0.0, g)
        h = np.where(near, h0, h1)
        u = np.where(near, u0, u1)
        return np.stack([h, h * u])
    return _cell_average(sampler, n, sub)


def euler_sod_exact(n: int, t: float, gamma=1.4, sub=16):
    """Cell averages of (rho, rho u, E) on n periodic cells for ``euler_sod``."""
    L = (1.0, 0.0, 1.0)
    R = (0.125, 0.0, 0.1)

    def sampler(x):
        near, xi = _periodic_xi(x, t)
        w0 = euler_sample(xi, *L, *R, gamma)
        w1 = euler_sample(xi, *R, *L, gamma)
        w = np.where(near[None, :], w0, w1)
        rho, u, p = w
        return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])
    return _cell_average(sampler, n, sub)
