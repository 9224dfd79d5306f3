"""FP64 oracle of the shallow-water bed-slope source term and of reflecting
walls (for both equations) (test infrastructure only).

Eq. 2.3 (and Section 4.2) add the source S = (0, -g h dz/dx, -g h dz/dy) of
a bed z(x, y) to the momentum equations; Section 4.2's bathymetry test runs
with wall boundaries instead of the periodic ones of every other test.  The
paper prints the PDE only.  Readings (each listed with its reason in the
design notes):
  * the bed is given at the cell centres and its slope is the centred
    difference (z_{i+1} - z_{i-1}) / (2 dx), (z_{j+1} - z_{j-1}) / (2 dy);
  * the source uses the depth h of the state the right-hand side is
    evaluated on (every Runge-Kutta stage), and is added to the flux
    divergence of that state: L(q) = -div F(q) + S(q, z);
  * a wall is a mirror: ghost cell k outside the domain copies the interior
    cell at the same distance from the wall, with the momentum normal to the
    wall negated (so the HLL mass flux through the wall vanishes); the bed
    is mirrored without a sign change.
With a bed that is linear in x and a flat water surface these choices
balance exactly away from the walls (MUSCL-minmod reconstructs linear data
exactly, the HLL diffusion terms vanish, and the centred slope times h_i
equals the pressure-flux difference); on other beds the balance holds to
second order in the mesh size.
"""
from __future__ import annotations

import torch

from . import fv
from . import schemes

PERIODIC = "periodic"
WALL = "wall"


def pad(q: torch.Tensor, dim: int, bc: str, n: int = 2, normal: int | None = None) -> torch.Tensor:
    """``q`` extended by ``n`` ghost cells on both ends of ``dim``: the
    periodic continuation, or (``WALL``) the mirror image with component
    ``normal`` of dim -3 negated (``None``: no sign change, for the bed)."""
    L = q.shape[dim]
    if bc == PERIODIC:
        lo = q.narrow(dim, L - n, n)
        hi = q.narrow(dim, 0, n)
    else:
        lo = q.narrow(dim, 0, n).flip(dim)
        hi = q.narrow(dim, L - n, n).flip(dim)
        if normal is not None:
            lo = lo.clone()
            hi = hi.clone()
            lo[..., normal, :, :] = -lo[..., normal, :, :]
            hi[..., normal, :, :] = -hi[..., normal, :, :]
    return torch.cat([lo, q, hi], dim=dim)


def muscl_faces(P: torch.Tensor, dim: int, delta: float):
    """MUSCL-minmod face states on a padded array (2 ghosts per end): the
    n + 1 faces from the west face of the first interior cell to the east
    face of the last, Q^L = Q_i + s_i dx / 2, Q^R = Q_{i+1} - s_{i+1} dx / 2
    with s = MINMOD((Q_i - Q_{i-1}) / dx, (Q_{i+1} - Q_i) / dx) (Eq. 2.18)."""
    m = P.shape[dim]
    Pm = P.narrow(dim, 0, m - 2)     # Q_{p-1}, p = 1 .. m-2
    P0 = P.narrow(dim, 1, m - 2)     # Q_p
    Pp = P.narrow(dim, 2, m - 2)     # Q_{p+1}
    slope = fv.minmod((P0 - Pm) / delta, (Pp - P0) / delta)
    ext_l = P0 + slope * delta / 2   # left state of the face p+1/2
    ext_r = P0 - slope * delta / 2   # right state of the face p-1/2
    k = m - 3                        # faces between padded cells p, p+1 for p = 1 .. m-3
    QL = ext_l.narrow(dim, 0, k)
    QR = ext_r.narrow(dim, 1, k)
    return QL, QR


def rhs(q: torch.Tensor, dx: float, dy: float, *, flux: str = schemes.HLL, z: torch.Tensor | None = None,
        bc: str = PERIODIC, dt=None, g: float = 9.81, eq: str = fv.SWE, gamma: float = 1.4) -> torch.Tensor:
    """L(q) on ``q`` [B][C][ny][nx] with the boundary ``bc`` on all four
    sides and, for shallow water, the bed ``z`` [ny][nx] (None: flat).  The
    momentum normal to a wall is component 1 (x) or 2 (y) for both
    equations."""
    nu_x = nu_y = None
    if flux == schemes.LAX_FRIEDRICHS:
        dt = torch.as_tensor(dt, dtype=q.dtype).reshape(-1)
        nu_x, nu_y = dx / (4.0 * dt), dy / (4.0 * dt)
    Px = pad(q, -1, bc, normal=1)
    QLx, QRx = muscl_faces(Px, -1, dx)
    Fx = schemes.face_flux(flux, QLx, QRx, *fv.X_FACE, eq, g, gamma, nu_x)   # nx + 1 faces
    Py = pad(q, -2, bc, normal=2)
    QLy, QRy = muscl_faces(Py, -2, dy)
    Gy = schemes.face_flux(flux, QLy, QRy, *fv.Y_FACE, eq, g, gamma, nu_y)   # ny + 1 faces
    F_w, F_e = Fx[..., :-1], Fx[..., 1:]
    G_s, G_n = Gy[..., :-1, :], Gy[..., 1:, :]
    L = -(dy * (F_e - F_w) + dx * (G_n - G_s)) / (dx * dy)
    if z is not None:
        zz = torch.as_tensor(z, dtype=q.dtype)[None, None]
        zx = pad(zz, -1, bc, n=1)
        zy = pad(zz, -2, bc, n=1)
        dzdx = (zx[..., 2:] - zx[..., :-2]) / (2.0 * dx)
        dzdy = (zy[..., 2:, :] - zy[..., :-2, :]) / (2.0 * dy)
        h = q[:, 0:1]
        L = L.clone()
        L[:, 1:2] = L[:, 1:2] - g * h * dzdx
        L[:, 2:3] = L[:, 2:3] - g * h * dzdy
    return L


def run(q0, nsteps: int, *, flux: str = schemes.HLL, rk: int = schemes.RK2, z=None, bc: str = PERIODIC,
        cfl: float = 0.5, dt_mode: str = fv.DT_ADAPTIVE, dt_fixed=None, dts=None, g: float = 9.81,
        eq: str = fv.SWE, gamma: float = 1.4, dtype=torch.float64):
    """``nsteps`` steps of the scheme with walls (and, for shallow water, a
    bed); the adaptive dt is the CFL rule of Eq. 2.10.  Returns (q, t,
    dt_history).  ``dtype`` float32 replays the same algorithm in single
    precision (the roundoff yardstick of the GPU parity tests)."""
    q = torch.as_tensor(q0).to(dtype).clone()
    B = q.shape[0]
    dx, dy = fv.grid_spacing(q)
    t = torch.zeros(B, dtype=dtype)
    hist = []
    for n in range(nsteps):
        if dt_mode == fv.DT_ADAPTIVE:
            dt = fv.cfl_dt(q, eq, cfl, dx, dy, g, gamma).to(dtype)
        elif dt_mode == fv.DT_FIXED:
            dt = torch.full((B,), float(dt_fixed), dtype=dtype)
        else:
            d = torch.as_tensor(dts[n]).to(dtype)
            dt = d.expand(B).clone() if d.dim() == 0 else d.clone()

        def L(s, dt=dt):
            return rhs(s, dx, dy, flux=flux, z=z, bc=bc, dt=dt, g=g, eq=eq, gamma=gamma)

        step = fv.ssp_rk2 if rk == schemes.RK2 else schemes.ssp_rk3
        q = step(q, dt.view(B, 1, 1, 1), L)
        t = t + dt
        hist.append(dt)
    dt_hist = torch.stack(hist) if hist else torch.zeros(0, B, dtype=dtype)
    return q, t, dt_hist
