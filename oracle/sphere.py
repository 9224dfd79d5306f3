"""FP64 oracle of the shallow-water equations on the sphere (test
infrastructure only).

Section 2.4 (the logically rectangular grid) and Section 4.3 (SWE on the
sphere).  The state is q = (h, hu, hv, hw) with a Cartesian momentum m in
R^3; the sphere has radius 1.

Grid.  The computational rectangle [-3, 1] x [-1, 1] carries nx x ny cells
(nx = 2 ny).  A point (xc, yc) with xc >= -1 lies on the upper hemisphere:
the disk mapping of Section 2.4 with D(d) = d / sqrt 2, R(d) = 1 gives
(xp, yp) and zp = sqrt(1 - xp^2 - yp^2) (Eq. 2.25); a point with xc < -1 is
the disk mapping of (-2 - xc, yc) with zp < 0.  The two disks meet along
xc = -1 (the equator), the rectangle is periodic in x (xc = -3 and xc = 1
are the same equator points), and its top (bottom) edge is glued to itself
reversed: the cell above (i, ny - 1) is (nx - 1 - i, ny - 1).

Discretisation (Section 4.3's steps 1-7):
  * edge lengths are great-circle distances between the edge's corners and
    cell areas spherical-quadrilateral areas (two spherical triangles);
  * at each edge t is the unit chord (second corner minus first), r the unit
    radial vector through the chord's midpoint, n = t x r oriented from the
    cell before the edge to the cell after it; (n, t, r) is orthonormal;
  * face states by MUSCL-minmod in the logical index directions (Eq. 2.18)
    on the Cartesian variables, rotated to (h, m.n, m.t, m.r), the HLL flux
    of the 1D problem in that frame (the r and t momenta are passive), and
    rotated back: F = (F0, F1 n + F2 t + F3 r);
  * L(q)_i = -(1 / A_i) [ sum_e l_e F_e.(+-) - F(q_i) . sum_e l_e n_e^out ]
    for the momenta (Eq. 3.1's correction: the discrete divergence of the
    cell's own flux, nonzero because the edge normals of a cell on the
    curved surface do not close, so that a lake at rest stays at rest); the
    depth keeps the plain flux difference, so mass is conserved exactly;
  * the Coriolis source of Eq. 3.2, -2 Omega z (x x m) with x the unit cell
    centre (the corner average normalised) and z its z coordinate, is added
    to L;
  * after every Runge-Kutta stage the momentum is projected onto the tangent
    plane at the cell centre, m <- m - (m.x) x (Eq. 3.2's second term);
  * dt by the Courant rate (|m| / h + sqrt(g h)) (sum_e l_e) / (2 A_i).
Fluxes other than HLL (Rusanov, Roe, HLLE, HLLC; Table 4 compares them on
the sphere) come from ``oracle.schemes``' shallow-water solvers applied to
(h, m.n, m.t) and to (h, m.n, m.r): both tangential momenta are passive, so
the second call's depth and normal fluxes equal the first's and its third
component is the flux of m.r.
"""
from __future__ import annotations

import math

import torch

from . import fv
from . import schemes

SQRT2 = math.sqrt(2.0)


def disk_map(xc: torch.Tensor, yc: torch.Tensor):
    """Section 2.4's mapping of the square [-1, 1]^2 onto the unit disk with
    D(d) = d / sqrt 2, R(d) = 1, sector by sector (|yc| <= |xc|: the arcs of
    the x sectors; otherwise the y sectors).  Returns (xp, yp, 1 - xp^2 -
    yp^2), the last written as -b (b + 2 s) with b = D - sqrt(1 - D^2) =
    (d^2 - 1) / (D + sqrt(1 - D^2)) and s the arc's square root, which is
    exact algebra and keeps its accuracy at the rim where it vanishes."""
    d = torch.maximum(xc.abs(), yc.abs())
    D = d / SQRT2
    safe = torch.where(d > 0, d, torch.ones_like(d))
    base = (d * d - 1.0) / (D + torch.sqrt(1.0 - D * D))
    xsec = yc.abs() <= xc.abs()
    # x sectors: y_p = y_c D / d, x_p = sign(x_c) (D - sqrt(1 - D^2) + sqrt(1 - y_p^2))
    yp_x = yc * D / safe
    s_x = torch.sqrt(1.0 - yp_x * yp_x)
    xp_x = torch.sign(xc) * (base + s_x)
    # y sectors: the same with the roles of x and y exchanged
    xp_y = xc * D / safe
    s_y = torch.sqrt(1.0 - xp_y * xp_y)
    yp_y = torch.sign(yc) * (base + s_y)
    xp = torch.where(xsec, xp_x, xp_y)
    yp = torch.where(xsec, yp_x, yp_y)
    sarc = torch.where(xsec, s_x, s_y)
    z2 = -base * (base + 2.0 * sarc)
    return xp, yp, z2


def sphere_point(xc: torch.Tensor, yc: torch.Tensor) -> torch.Tensor:
    """Points [..., 3] on the unit sphere for computational coordinates in
    [-3, 1] x [-1, 1] (upper hemisphere for xc >= -1)."""
    upper = xc >= -1.0
    xd = torch.where(upper, xc, -2.0 - xc)
    xp, yp, z2 = disk_map(xd, yc)
    zp = torch.sqrt(torch.clamp(z2, min=0.0))
    zp = torch.where(upper, zp, -zp)
    return torch.stack([xp, yp, zp], dim=-1)


def corners(nx: int, ny: int) -> torch.Tensor:
    """Cell corners P[ny + 1][nx + 1][3].  Each hemisphere's square is
    sampled at s_k = (2 k - ny) / ny, k = 0..ny (so s_{ny - k} = -s_k
    exactly): upper-block corner column k is the disk point (s_k, s_j), and
    lower-block column k (xc = -3 + 2 k / ny) is the disk point (-s_k, s_j)
    below the equator, which makes the glued corners bitwise equal."""
    k = torch.arange(ny + 1, dtype=torch.float64)
    s = (2.0 * k - ny) / ny
    Y, X = torch.meshgrid(s, s, indexing="ij")
    xu, yu, zu = disk_map(X, Y)
    xl, yl, zl = disk_map(-X, Y)
    up = torch.stack([xu, yu, torch.sqrt(torch.clamp(zu, min=0.0))], dim=-1)
    lo = torch.stack([xl, yl, -torch.sqrt(torch.clamp(zl, min=0.0))], dim=-1)
    return torch.cat([lo[:, :ny], up], dim=1)


def _unit(v: torch.Tensor) -> torch.Tensor:
    return v / v.norm(dim=-1, keepdim=True)


def great_circle(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Great-circle distance on the unit sphere, 2 asin(|a - b| / 2)."""
    return 2.0 * torch.asin(torch.clamp((a - b).norm(dim=-1) / 2.0, max=1.0))


def triangle_area(a, b, c) -> torch.Tensor:
    """Spherical excess of the triangle abc on the unit sphere:
    tan(E / 2) = |a . (b x c)| / (1 + a.b + b.c + c.a)."""
    num = (a * torch.cross(b, c, dim=-1)).sum(-1).abs()
    den = 1.0 + (a * b).sum(-1) + (b * c).sum(-1) + (c * a).sum(-1)
    return 2.0 * torch.atan2(num, den)


class Grid:
    """Metrics of the nx x ny sphere grid (FP64)."""

    def __init__(self, nx: int, ny: int):
        assert nx == 2 * ny and ny >= 2
        self.nx, self.ny = nx, ny
        P = corners(nx, ny)
        self.P = P
        p00, p10, p01, p11 = P[:-1, :-1], P[:-1, 1:], P[1:, :-1], P[1:, 1:]
        self.area = triangle_area(p00, p10, p11) + triangle_area(p00, p11, p01)        # [ny][nx]
        self.centre = _unit(p00 + p10 + p01 + p11)                                   # [ny][nx][3]
        # x faces: face i between cells i - 1 and i, corners P[j][i] -> P[j + 1][i]; i = 0..nx - 1
        a, b = P[:-1, :-1], P[1:, :-1]
        self.fx_len = great_circle(a, b)
        t = _unit(b - a)
        r = _unit(a + b)
        n = torch.cross(t, r, dim=-1)
        right = self.centre
        left = torch.roll(self.centre, 1, dims=1)
        s = torch.sign(((right - left) * n).sum(-1, keepdim=True))
        self.fx_n, self.fx_t, self.fx_r = n * s, t, r
        # y faces: face j between rows j - 1 and j, corners P[j][i] -> P[j][i + 1]; j = 0..ny
        a, b = P[:, :-1], P[:, 1:]
        self.fy_len = great_circle(a, b)
        t = _unit(b - a)
        r = _unit(a + b)
        n = torch.cross(t, r, dim=-1)
        c_pad = self.pad_y(self.centre.permute(2, 0, 1).unsqueeze(0), 1)[0].permute(1, 2, 0)
        below, above = c_pad[:-1], c_pad[1:]                                          # rows j - 1, j
        s = torch.sign(((above - below) * n).sum(-1, keepdim=True))
        self.fy_n, self.fy_t, self.fy_r = n * s, t, r
        # sum of l_e n_e over each cell's edges, outward
        self.ln_sum = (torch.roll(self.fx_len[..., None] * self.fx_n, -1, dims=1) - self.fx_len[..., None] * self.fx_n
                       + self.fy_len[1:, :, None] * self.fy_n[1:] - self.fy_len[:-1, :, None] * self.fy_n[:-1])
        self.perimeter = (self.fx_len + torch.roll(self.fx_len, -1, dims=1) + self.fy_len[1:] + self.fy_len[:-1])

    def pad_y(self, q: torch.Tensor, n: int = 2) -> torch.Tensor:
        """q [..., ny, nx] with n ghost rows on each side: above row ny - 1
        the rows ny - 1, ny - 2, ... of the mirrored columns, below row 0 the
        rows 0, 1, ... of the mirrored columns."""
        top = q[..., -n:, :].flip(-2).flip(-1)
        bot = q[..., :n, :].flip(-2).flip(-1)
        return torch.cat([bot, q, top], dim=-2)


def hll4(qL: torch.Tensor, qR: torch.Tensor, g: float) -> torch.Tensor:
    """HLL flux (Eq. 2.15) of two face-frame states (h, m_n, m_t, m_r) [B][4][...]:
    the normal flux (m_n, m_n^2 / h + g h^2 / 2, m_n m_t / h, m_n m_r / h)."""
    def phys(q):
        h, mn = q[:, 0], q[:, 1]
        un = mn / h
        return torch.stack([mn, mn * un + 0.5 * g * h * h, q[:, 2] * un, q[:, 3] * un], dim=1), un, torch.sqrt(g * h)
    FL, uL, cL = phys(qL)
    FR, uR, cR = phys(qR)
    sL = torch.minimum(uL - cL, uR - cR).unsqueeze(1)
    sR = torch.maximum(uL + cL, uR + cR).unsqueeze(1)
    F = (sR * FL - sL * FR + sL * sR * (qR - qL)) / (sR - sL)
    return torch.where(sL >= 0, FL, torch.where(sR < 0, FR, F))


def rotate(q: torch.Tensor, n, t, r) -> torch.Tensor:
    """(h, m.n, m.t, m.r) of q [B][4][...] with frame vectors [..., 3]."""
    m = q[:, 1:4]
    def dot(v):
        return (m * v.movedim(-1, 0).unsqueeze(0)).sum(1)
    return torch.stack([q[:, 0], dot(n), dot(t), dot(r)], dim=1)


def rotate_back(f: torch.Tensor, n, t, r) -> torch.Tensor:
    vn, vt, vr = (v.movedim(-1, 0).unsqueeze(0) for v in (n, t, r))
    m = f[:, 1:2] * vn + f[:, 2:3] * vt + f[:, 3:4] * vr
    return torch.cat([f[:, :1], m], dim=1)


def flux_dot(q: torch.Tensor, S: torch.Tensor, g: float) -> torch.Tensor:
    """F(q) . S for a vector S [..., 3]: (m.S, m (m.S) / h + (g h^2 / 2) S)."""
    h, m = q[:, 0], q[:, 1:4]
    Sv = S.movedim(-1, 0).unsqueeze(0)
    mS = (m * Sv).sum(1)
    mom = m * (mS / h).unsqueeze(1) + (0.5 * g * h * h).unsqueeze(1) * Sv
    return torch.cat([mS.unsqueeze(1), mom], dim=1)


def edge_flux(flux: str, qL: torch.Tensor, qR: torch.Tensor, g: float) -> torch.Tensor:
    """Normal flux of two edge-frame states (h, m_n, m_t, m_r) [B][4][...]."""
    if flux == schemes.HLL:
        return hll4(qL, qR, g)
    a = schemes.normal_flux_solver(flux, qL[:, :3], qR[:, :3], fv.SWE, g, 1.4)
    b = schemes.normal_flux_solver(flux, qL[:, [0, 1, 3]], qR[:, [0, 1, 3]], fv.SWE, g, 1.4)
    return torch.cat([a, b[:, 2:3]], dim=1)


def rhs(q: torch.Tensor, G: Grid, g: float, omega: float, flux: str = schemes.HLL) -> torch.Tensor:
    """L(q) for q [B][4][ny][nx]."""
    # x faces (periodic): face i between cells i - 1 and i
    QL, QR = fv.muscl_minmod(q, -1, 1.0)          # face i + 1/2 at index i (slopes in index units)
    QL = torch.roll(QL, 1, dims=-1)                # now face i (left cell i - 1)
    QR = torch.roll(QR, 1, dims=-1)
    Fx = rotate_back(edge_flux(flux, rotate(QL, G.fx_n, G.fx_t, G.fx_r), rotate(QR, G.fx_n, G.fx_t, G.fx_r), g),
                     G.fx_n, G.fx_t, G.fx_r) * G.fx_len
    # y faces: face j between rows j - 1 and j, j = 0..ny, from the padded array
    P = G.pad_y(q, 2)
    m = P.shape[-2]
    Pm, P0, Pp = P[..., :m - 2, :], P[..., 1:m - 1, :], P[..., 2:, :]
    slope = fv.minmod(P0 - Pm, Pp - P0)
    up = P0 + 0.5 * slope          # upper face state of padded rows 1..m-2
    dn = P0 - 0.5 * slope          # lower face state
    QL = up[..., :-1, :]           # rows -1 .. ny - 1  (face j's lower cell j - 1)
    QR = dn[..., 1:, :]            # rows 0 .. ny
    Gy = rotate_back(edge_flux(flux, rotate(QL, G.fy_n, G.fy_t, G.fy_r), rotate(QR, G.fy_n, G.fy_t, G.fy_r), g),
                     G.fy_n, G.fy_t, G.fy_r) * G.fy_len
    net = (torch.roll(Fx, -1, dims=-1) - Fx) + (Gy[..., 1:, :] - Gy[..., :-1, :])
    corr = flux_dot(q, G.ln_sum, g)
    corr[:, 0] = 0.0                     # the depth equation stays conservative
    L = -(net - corr) / G.area
    # Coriolis: -2 Omega z (x cross m)
    x = G.centre.movedim(-1, 0).unsqueeze(0)
    cor = -2.0 * omega * x[:, 2:3] * torch.cross(x.expand_as(q[:, 1:4]), q[:, 1:4], dim=1)
    L = L.clone()
    L[:, 1:4] = L[:, 1:4] + cor
    return L


def project(q: torch.Tensor, G: Grid) -> torch.Tensor:
    """Momentum onto the tangent plane at each cell centre."""
    x = G.centre.movedim(-1, 0).unsqueeze(0)
    m = q[:, 1:4]
    m = m - (m * x).sum(1, keepdim=True) * x
    return torch.cat([q[:, :1], m], dim=1)


def step(q: torch.Tensor, G: Grid, dt, g: float, omega: float, flux: str = schemes.HLL) -> torch.Tensor:
    """SSP-RK2 (Eq. 2.19) with the tangent projection after each stage."""
    q1 = project(q + dt * rhs(q, G, g, omega, flux), G)
    return project(0.5 * q + 0.5 * q1 + 0.5 * dt * rhs(q1, G, g, omega, flux), G)


def cfl_dt(q: torch.Tensor, G: Grid, cfl: float, g: float) -> torch.Tensor:
    h = q[:, 0]
    speed = q[:, 1:4].norm(dim=1) / h + torch.sqrt(g * h)
    rate = speed * G.perimeter / (2.0 * G.area)
    return cfl / rate.amax(dim=(-1, -2))


def run(q0, G: Grid, nsteps: int, *, g: float, omega: float, cfl: float = 0.5,
        dt_mode: str = fv.DT_ADAPTIVE, dt_fixed=None, dts=None, dtype=torch.float64, flux: str = schemes.HLL):
    """``nsteps`` SSP-RK2 steps; returns (q, t, dt_history).  ``dtype``
    float32 replays the algorithm in single precision (metrics included)."""
    q = torch.as_tensor(q0).to(dtype).clone()
    if dtype != torch.float64:
        G = _cast(G, dtype)
    B = q.shape[0]
    t = torch.zeros(B, dtype=dtype)
    hist = []
    for n in range(nsteps):
        if dt_mode == fv.DT_ADAPTIVE:
            dt = cfl_dt(q, G, cfl, g).to(dtype)
        elif dt_mode == fv.DT_FIXED:
            dt = torch.full((B,), float(dt_fixed), dtype=dtype)
        else:
            d = torch.as_tensor(dts[n]).to(dtype)
            dt = d.expand(B).clone() if d.dim() == 0 else d.clone()
        q = step(q, G, dt.view(B, 1, 1, 1), g, omega, flux)
        t = t + dt
        hist.append(dt)
    dt_hist = torch.stack(hist) if hist else torch.zeros(0, B, dtype=torch.float64)
    return q, t, dt_hist


def _cast(G: Grid, dtype) -> Grid:
    H = Grid.__new__(Grid)
    for k, v in vars(G).items():
        setattr(H, k, v.to(dtype) if torch.is_tensor(v) else v)
    return H


def mass(q: torch.Tensor, G: Grid) -> torch.Tensor:
    """Total mass sum_i A_i h_i per member."""
    return (q[:, 0] * G.area).sum(dim=(-1, -2))
