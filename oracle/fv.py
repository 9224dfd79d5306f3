"""FP64 oracle of the plain finite-volume step (test infrastructure only).

State layout: ``q[B][C][ny][nx]`` float64, x along the last axis, periodic.
SWE: C = 3, q = (h, hu, hv)   (Eq. 2.3 with a flat bed, S = 0).
Euler: C = 4, q = (rho, rho u, rho v, E) with the ideal-gas law (Eq. 2.4 in
its 2D form p = (gamma - 1)(E - rho (u^2 + v^2) / 2)), Section 4.2.

One right-hand side L(q) (Section 2.3.4, steps 1-5):
  1. reconstruct face states by MUSCL-minmod (Eq. 2.18),
  2. rotate each face's states into its normal frame (Eq. 2.24),
  3. numerical flux by HLL (Eq. 2.15),
  4. rotate the flux back (R^T),
  5. conservative update of every cell from the fluxes through its sides
     (Eq. 2.23 with side length h_i and cell area dc = dx dy).
Time integration is Heun / SSP-RK2 (Eq. 2.19); dt follows the CFL rule
(Eq. 2.10).

Readings of the paper where it is garbled or silent (each one is listed with
its reason in the design notes):
  * MINMOD's second branch prints "|b| < |b|"; read |b| < |a|.
  * Q^R_{i+1/2} prints "+ MINMOD(...) dx/2"; read "-": it extrapolates cell
    i+1 to its own left face.  Only this reading reproduces linear data.
  * Reconstruction acts on the conserved variables, component-wise.
  * HLL's lambda_L, lambda_R are undefined; we take the Davis estimates
    s_L = min(u_L - c_L, u_R - c_R), s_R = max(u_L + c_L, u_R + c_R) with u
    the face-normal velocity of the reconstructed states.
  * The grid has N cells of width 1/N (the printed N+1 indexing is garbled).
  * Adaptive dt from the 2D Courant number of the unsplit update:
    dt = CFL / max_cells((|u| + c)/dx + (|v| + c)/dy), evaluated on q^n and
    held for both stages (Eq. 2.10 extended to two directions).
"""
from __future__ import annotations

import torch

SWE = "swe"
EULER = "euler"

DT_ADAPTIVE = "adaptive"
DT_FIXED = "fixed"
DT_REPLAY = "replay"


# ----------------------------------------------------------------------------
# Physics: normal-frame flux and wave speed (Eqs. 2.3, 2.4, 2.5; Section 4.2)
# ----------------------------------------------------------------------------

def pressure(q: torch.Tensor, gamma: float) -> torch.Tensor:
    """Ideal-gas pressure p = (gamma - 1)(E - rho (u^2 + v^2)/2) (Eq. 2.4, 2D)."""
    rho, mu, mv, E = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return (gamma - 1.0) * (E - 0.5 * (mu * mu + mv * mv) / rho)


def normal_flux(qn: torch.Tensor, eq: str, g: float, gamma: float) -> torch.Tensor:
    """x-direction physical flux of a state already rotated into the face
    frame (component 1 = normal momentum, component 2 = tangential)."""
    if eq == SWE:
        h, m, t = qn[:, 0], qn[:, 1], qn[:, 2]
        u = m / h
        return torch.stack([m, m * u + 0.5 * g * h * h, t * u], dim=1)
    rho, m, t, E = qn[:, 0], qn[:, 1], qn[:, 2], qn[:, 3]
    u = m / rho
    p = pressure(qn, gamma)
    return torch.stack([m, m * u + p, t * u, u * (E + p)], dim=1)


def normal_velocity_and_sound_speed(qn: torch.Tensor, eq: str, g: float, gamma: float):
    """(u_n, c): c = sqrt(g h) for SWE, c = sqrt(gamma p / rho) for Euler."""
    if eq == SWE:
        h = qn[:, 0]
        return qn[:, 1] / h, torch.sqrt(g * h)
    rho = qn[:, 0]
    return qn[:, 1] / rho, torch.sqrt(gamma * pressure(qn, gamma) / rho)


# ----------------------------------------------------------------------------
# Eq. 2.24: rotation into the face frame and back
# ----------------------------------------------------------------------------

def rotate(q: torch.Tensor, n, t) -> torch.Tensor:
    """q_bullet = R q with R = [[1,0,0],[0,n1,n2],[0,t1,t2]] acting on the
    momentum pair; the other components are untouched."""
    out = q.clone()
    out[:, 1] = n[0] * q[:, 1] + n[1] * q[:, 2]
    out[:, 2] = t[0] * q[:, 1] + t[1] * q[:, 2]
    return out


def rotate_back(f: torch.Tensor, n, t) -> torch.Tensor:
    """F = R^T F_bullet."""
    out = f.clone()
    out[:, 1] = n[0] * f[:, 1] + t[0] * f[:, 2]
    out[:, 2] = n[1] * f[:, 1] + t[1] * f[:, 2]
    return out


# ----------------------------------------------------------------------------
# Eq. 2.15: HLL numerical flux in the face frame
# ----------------------------------------------------------------------------

def hll(qL: torch.Tensor, qR: torch.Tensor, eq: str, g: float, gamma: float) -> torch.Tensor:
    """Three-branch HLL flux of two face-frame states."""
    uL, cL = normal_velocity_and_sound_speed(qL, eq, g, gamma)
    uR, cR = normal_velocity_and_sound_speed(qR, eq, g, gamma)
    sL = torch.minimum(uL - cL, uR - cR).unsqueeze(1)
    sR = torch.maximum(uL + cL, uR + cR).unsqueeze(1)
    FL = normal_flux(qL, eq, g, gamma)
    FR = normal_flux(qR, eq, g, gamma)
    F_hll = (sR * FL - sL * FR + sL * sR * (qR - qL)) / (sR - sL)
    return torch.where(sL >= 0, FL, torch.where(sR < 0, FR, F_hll))


def face_flux(qL: torch.Tensor, qR: torch.Tensor, n, t, eq: str, g: float,
              gamma: float) -> torch.Tensor:
    """Section 2.3.4 steps 1-3: rotate, solve the 1D problem, rotate back."""
    return rotate_back(hll(rotate(qL, n, t), rotate(qR, n, t), eq, g, gamma), n, t)


X_FACE = ((1.0, 0.0), (0.0, 1.0))    # (n, t) of a face normal to +x
Y_FACE = ((0.0, 1.0), (-1.0, 0.0))   # (n, t) of a face normal to +y


# ----------------------------------------------------------------------------
# Eq. 2.18: MUSCL reconstruction with the MINMOD limiter
# ----------------------------------------------------------------------------

def minmod(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """a if |a| < |b| and ab > 0; b if |b| <= |a| and ab > 0; 0 if ab <= 0."""
    return torch.where(a * b <= 0, torch.zeros_like(a),
                       torch.where(a.abs() < b.abs(), a, b))


def muscl_minmod(Q: torch.Tensor, dim: int, delta: float):
    """Face states at i+1/2 (stored at index i) along ``dim``:
    Q^L_{i+1/2} = Q_i + MINMOD((Q_i - Q_{i-1})/dx, (Q_{i+1} - Q_i)/dx) dx/2,
    Q^R_{i+1/2} = Q_{i+1} - MINMOD((Q_{i+1} - Q_i)/dx, (Q_{i+2} - Q_{i+1})/dx) dx/2.
    """
    Qm = torch.roll(Q, 1, dims=dim)    # Q_{i-1}
    Qp = torch.roll(Q, -1, dims=dim)   # Q_{i+1}
    slope = minmod((Q - Qm) / delta, (Qp - Q) / delta)
    QL = Q + slope * delta / 2
    QR = torch.roll(Q - slope * delta / 2, -1, dims=dim)
    return QL, QR


def first_order_faces(Q: torch.Tensor, dim: int):
    """Piecewise-constant reconstruction: Q^L_{i+1/2} = Q_i, Q^R = Q_{i+1}."""
    return Q.clone(), torch.roll(Q, -1, dims=dim)


# ----------------------------------------------------------------------------
# Section 2.3.4 / Eq. 2.23: the semi-discrete right-hand side
# ----------------------------------------------------------------------------

def divergence_update(F: torch.Tensor, G: torch.Tensor, dx: float, dy: float) -> torch.Tensor:
    """-(1/dc) sum_sides h_i Fbar_i for a Cartesian cell: east/west sides of
    length dy carry F_{i+1/2}, -F_{i-1/2}; north/south sides of length dx carry
    G_{j+1/2}, -G_{j-1/2}; dc = dx dy.  F, G are stored at face i+1/2 / j+1/2."""
    dc = dx * dy
    side_sum = dy * (F - torch.roll(F, 1, dims=-1)) + dx * (G - torch.roll(G, 1, dims=-2))
    return -side_sum / dc


def rhs(q: torch.Tensor, eq: str, dx: float, dy: float, g: float = 9.81,
        gamma: float = 1.4, recon=None) -> torch.Tensor:
    """L(q) for the whole periodic grid.  ``recon(Q, dim, delta)`` returns the
    (Q^L, Q^R) face states; MUSCL-minmod by default."""
    recon = recon or muscl_minmod
    QLx, QRx = recon(q, -1, dx)
    F = face_flux(QLx, QRx, *X_FACE, eq, g, gamma)
    QLy, QRy = recon(q, -2, dy)
    G = face_flux(QLy, QRy, *Y_FACE, eq, g, gamma)
    return divergence_update(F, G, dx, dy)


def ssp_rk2(q: torch.Tensor, dt, L) -> torch.Tensor:
    """Heun / SSP-RK2 (Eq. 2.19): q1 = q + dt L(q); q' = q/2 + q1/2 + dt L(q1)/2."""
    q1 = q + dt * L(q)
    return 0.5 * q + 0.5 * q1 + 0.5 * dt * L(q1)


# ----------------------------------------------------------------------------
# Eq. 2.10: CFL time step
# ----------------------------------------------------------------------------

def max_courant_rate(q: torch.Tensor, eq: str, dx: float, dy: float, g: float = 9.81,
                     gamma: float = 1.4) -> torch.Tensor:
    """Per member: max over cells of (|u| + c)/dx + (|v| + c)/dy, the rate at
    which the 2D Courant number of the unsplit update grows with dt."""
    if eq == SWE:
        h = q[:, 0]
        u, v, c = q[:, 1] / h, q[:, 2] / h, torch.sqrt(g * h)
    else:
        rho = q[:, 0]
        u, v = q[:, 1] / rho, q[:, 2] / rho
        c = torch.sqrt(gamma * pressure(q, gamma) / rho)
    rate = (u.abs() + c) / dx + (v.abs() + c) / dy
    return rate.flatten(1).amax(dim=1)


def cfl_dt(q: torch.Tensor, eq: str, cfl: float, dx: float, dy: float,
           g: float = 9.81, gamma: float = 1.4) -> torch.Tensor:
    """dt per member such that the 2D Courant number
    C = dt * max_cells((|u| + c)/dx + (|v| + c)/dy) equals ``cfl``.

    Eq. 2.10 defines C = a dt / dx for one direction.  The update of Eq. 2.23
    takes all sides of a cell in one unsplit step, whose Courant number is the
    sum of the directional ones; with the per-direction reading at C = 0.5 the
    scheme amplifies grid-scale perturbations (C_x + C_y reaches 1)."""
    return cfl / max_courant_rate(q, eq, dx, dy, g, gamma)


# ----------------------------------------------------------------------------
# Driver
# ----------------------------------------------------------------------------

def grid_spacing(q: torch.Tensor, lx: float = 1.0, ly: float = 1.0):
    return lx / q.shape[-1], ly / q.shape[-2]


def run(q0, eq: str, nsteps: int, *, cfl: float = 0.5, dt_mode: str = DT_ADAPTIVE,
        dt_fixed: float | None = None, dts=None, g: float = 9.81, gamma: float = 1.4,
        lx: float = 1.0, ly: float = 1.0, recon=None, snapshot_every: int = 0):
    """Advance ``q0`` (``[B][C][ny][nx]``) by ``nsteps`` SSP-RK2 steps.

    dt_mode: "adaptive" (Eq. 2.10 on q^n, per member), "fixed" (``dt_fixed``)
    or "replay" (``dts[n]`` for step n, shared by all members, or ``[n][B]``).
    Returns ``(q, t, dt_history[nsteps][B], snapshots)``.
    """
    q = torch.as_tensor(q0, dtype=torch.float64).clone()
    B = q.shape[0]
    dx, dy = grid_spacing(q, lx, ly)
    t = torch.zeros(B, dtype=torch.float64)
    hist = []
    snaps = [q.clone()] if snapshot_every else []

    def L(s):
        return rhs(s, eq, dx, dy, g, gamma, recon)

    for n in range(nsteps):
        if dt_mode == DT_ADAPTIVE:
            dt = cfl_dt(q, eq, cfl, dx, dy, g, gamma)
        elif dt_mode == DT_FIXED:
            dt = torch.full((B,), float(dt_fixed), dtype=torch.float64)
        else:
            d = torch.as_tensor(dts[n], dtype=torch.float64)
            dt = d.expand(B).clone() if d.dim() == 0 else d.clone()
        q = ssp_rk2(q, dt.view(B, 1, 1, 1), L)
        t = t + dt
        hist.append(dt)
        if snapshot_every and (n + 1) % snapshot_every == 0:
            snaps.append(q.clone())
    dt_hist = torch.stack(hist) if hist else torch.zeros(0, B, dtype=torch.float64)
    return q, t, dt_hist, snaps


# ----------------------------------------------------------------------------
# Diagnostics (Section 5, Eq. 5.1) and coarse graining (Section 2.5.1)
# ----------------------------------------------------------------------------

def diagnostics(q: torch.Tensor, eq: str, g: float = 9.81, gamma: float = 1.4,
                lx: float = 1.0, ly: float = 1.0) -> torch.Tensor:
    """Per member ``[C + 1]``: the integral of every conserved variable over
    the domain (sum of cell averages times the cell area), then
    SWE: total energy, integral of g h^2 / 2 + (u^2 + v^2) h / 2 (Eq. 5.1);
    Euler: total kinetic energy, integral of rho (u^2 + v^2) / 2."""
    dx, dy = grid_spacing(q, lx, ly)
    area = dx * dy
    sums = [q[:, c].flatten(1).sum(dim=1) * area for c in range(q.shape[1])]
    if eq == SWE:
        h = q[:, 0]
        u, v = q[:, 1] / h, q[:, 2] / h
        e = 0.5 * g * h * h + 0.5 * (u * u + v * v) * h
    else:
        rho = q[:, 0]
        u, v = q[:, 1] / rho, q[:, 2] / rho
        e = 0.5 * rho * (u * u + v * v)
    sums.append(e.flatten(1).sum(dim=1) * area)
    return torch.stack(sums, dim=1)


def potential_enstrophy(q: torch.Tensor, lx: float = 1.0, ly: float = 1.0) -> torch.Tensor:
    """Planar potential enstrophy (f = 0): integral of zeta^2 / (2 h), with
    zeta = dv/dx - du/dy from centred differences of u = hu/h, v = hv/h.
    The paper names this diagnostic without defining it; this is the usual
    definition."""
    dx, dy = grid_spacing(q, lx, ly)
    h = q[:, 0]
    u, v = q[:, 1] / h, q[:, 2] / h
    dvdx = (torch.roll(v, -1, -1) - torch.roll(v, 1, -1)) / (2 * dx)
    dudy = (torch.roll(u, -1, -2) - torch.roll(u, 1, -2)) / (2 * dy)
    zeta = dvdx - dudy
    return (0.5 * zeta * zeta / h).flatten(1).sum(dim=1) * dx * dy


def coarsen(q: torch.Tensor, factor: int) -> torch.Tensor:
    """Block average of factor x factor fine cells: the coarse cell average."""
    B, C, ny, nx = q.shape
    return q.reshape(B, C, ny // factor, factor, nx // factor, factor).mean(dim=(3, 5))


def relative_errors(a: torch.Tensor, ref: torch.Tensor) -> dict:
    """Per variable: relative L2 = ||a - ref||_2 / ||ref||_2 and relative Linf
    = max|a - ref| / max|ref| (a variable that is identically zero in ``ref``
    is normalised by the largest magnitude of the first variable instead)."""
    out = {}
    scale0 = ref[:, 0].abs().max()
    for c in range(ref.shape[1]):
        d = (a[:, c] - ref[:, c])
        n2 = ref[:, c].norm()
        ninf = ref[:, c].abs().max()
        if float(ninf) == 0.0:
            n2 = scale0 * (ref[:, c].numel() ** 0.5)
            ninf = scale0
        out[c] = (float(d.norm() / n2), float(d.abs().max() / ninf))
    return out


def mean_relative_h_error(h_low: torch.Tensor, h_high: torch.Tensor) -> float:
    """Section 3 error metric, taken in absolute value: mean over cells of
    |h_high - h_low| / h_high."""
    return float(((h_high - h_low).abs() / h_high).mean())
