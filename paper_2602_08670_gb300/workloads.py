"""Seeded synthetic inputs: initial states and request streams.

This module only *builds inputs*.  It holds none of the scheme's arithmetic
(no reconstruction, no flux, no time step) and imports nothing else from this
package, so both the CUDA path and the FP64 CPU oracle draw their inputs from
it without depending on one another.

Every generator returns float64 numpy arrays in the state layout used across
the project: ``q[B][C][ny][nx]`` (x fastest), cell-centre point values on the
periodic unit square with ``N`` cells per direction and centres at
``(i + 1/2) * dx`` (Section 2.3.1, "The grid", read with N cells and dx = 1/N).
C = 3 for shallow water ``(h, hu, hv)`` and C = 4 for Euler
``(rho, rho*u, rho*v, E)``.

Randomness comes from numpy's Philox counter-based generator, seeded
explicitly, so a workload is reproducible from its seed alone.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

G_GRAVITY = 9.81      # g used by every shallow-water workload
GAMMA_IDEAL = 1.4     # ratio of specific heats for every Euler workload


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def cell_centres(n: int, length: float = 1.0) -> np.ndarray:
    """Centres x_i = (i + 1/2) * length / n, i = 0..n-1."""
    return (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def _mesh(nx: int, ny: int):
    x = cell_centres(nx)
    y = cell_centres(ny)
    return np.meshgrid(x, y, indexing="xy")  # X[j, i], Y[j, i]


def swe_gaussian_bump(nx: int, ny: int, amp: float = 0.1, width2: float = 0.005,
                      h0: float = 1.0) -> np.ndarray:
    """Shallow water at rest with a centred Gaussian hump.

    h = h0 + amp * exp(-((x-1/2)^2 + (y-1/2)^2) / width2), hu = hv = 0.
    With the defaults this is the 128x128 oracle workload and the 4096x4096
    throughput workload.  Returns ``[1][3][ny][nx]``.
    """
    X, Y = _mesh(nx, ny)
    h = h0 + amp * np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / width2)
    q = np.zeros((1, 3, ny, nx))
    q[0, 0] = h
    return q


def euler_kelvin_helmholtz(nx: int, ny: int, seed: int = 0,
                           gamma: float = GAMMA_IDEAL) -> np.ndarray:
    """Kelvin-Helmholtz shear layer for 2D Euler.

    Inner strip 1/4 <= y < 3/4: rho = 2, u = +0.5; outside: rho = 1, u = -0.5.
    v = 0.01 sin(4 pi x) + 1e-3 U(-1, 1) (seeded), uniform pressure p = 2.5.
    Returns conserved variables ``[1][4][ny][nx]`` with
    E = p / (gamma - 1) + rho (u^2 + v^2) / 2.
    """
    X, Y = _mesh(nx, ny)
    inner = (Y >= 0.25) & (Y < 0.75)
    rho = np.where(inner, 2.0, 1.0)
    u = np.where(inner, 0.5, -0.5)
    noise = _rng(seed).uniform(-1.0, 1.0, size=(ny, nx))
    v = 0.01 * np.sin(4.0 * math.pi * X) + 1e-3 * noise
    p = np.full_like(rho, 2.5)
    q = np.zeros((1, 4, ny, nx))
    q[0, 0] = rho
    q[0, 1] = rho * u
    q[0, 2] = rho * v
    q[0, 3] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return q


@dataclasses.dataclass
class BumpSpec:
    centres: np.ndarray   # [K, 2]
    amps: np.ndarray      # [K]
    widths: np.ndarray    # [K]


def random_bump_specs(seed: int, members: int) -> list[BumpSpec]:
    """Draw, per member, K ~ U{1..5} bumps with A ~ U[0.05, 0.2],
    w ~ U[0.02, 0.1] and centres ~ U[0, 1)^2."""
    rng = _rng(seed)
    out = []
    for _ in range(members):
        k = int(rng.integers(1, 6))
        out.append(BumpSpec(centres=rng.uniform(0.0, 1.0, size=(k, 2)),
                            amps=rng.uniform(0.05, 0.2, size=k),
                            widths=rng.uniform(0.02, 0.1, size=k)))
    return out


def swe_random_bumps(n: int, seed: int, members: int) -> np.ndarray:
    """Training / ensemble initial states: h = 1 + sum_k A_k exp(-d_k^2 / w_k^2),
    d_k the periodic minimum-image distance to centre k, hu = hv = 0.

    The same seed gives the same bumps at every resolution, so a 256x256 run
    and its 64x64 coarse counterpart start from the same continuous field.
    Returns ``[members][3][n][n]``.
    """
    X, Y = _mesh(n, n)
    q = np.zeros((members, 3, n, n))
    for b, spec in enumerate(random_bump_specs(seed, members)):
        h = np.ones((n, n))
        for (cx, cy), a, w in zip(spec.centres, spec.amps, spec.widths):
            dx = np.abs(X - cx)
            dx = np.minimum(dx, 1.0 - dx)
            dy = np.abs(Y - cy)
            dy = np.minimum(dy, 1.0 - dy)
            h += a * np.exp(-(dx * dx + dy * dy) / (w * w))
        q[b, 0] = h
    return q


def _gauss_cell_means(edges: np.ndarray, c: np.ndarray, w: np.ndarray) -> np.ndarray:
    """[K][n] means over the cells [edges[i], edges[i+1]) of the 1-periodic
    Gaussians exp(-(x - c_k)^2 / w_k^2) (images at -1, 0, +1)."""
    from scipy.special import erf
    h = edges[1:] - edges[:-1]
    out = np.zeros((len(c), len(edges) - 1))
    for k in (-1.0, 0.0, 1.0):
        z = (edges[None, :] - c[:, None] - k) / w[:, None]
        e = erf(z)
        out += (0.5 * math.sqrt(math.pi) * w[:, None]) * (e[:, 1:] - e[:, :-1])
    return out / h[None, :]


def swe_random_bumps_tiled(n: int, seed: int, members: int, tiles: int, first: int = 0) -> np.ndarray:
    """The training recipe with its features scaled to a finer grid: the unit
    square is cut into tiles x tiles squares of side 1/tiles, and each square
    gets its own draw of the random-bump recipe (K ~ U{1..5} bumps,
    A ~ U[0.05, 0.2], widths U[0.02, 0.1] / tiles, centres uniform in the
    square), h = 1 + sum_k A_k exp(-|x - c_k|^2 / w_k^2) with periodic images,
    fluid at rest.  The shallow-water equations on a flat bed have no length
    scale of their own (x -> x / t with time -> time / t leaves them
    unchanged), so an n^2 run of this field is locally the same problem as an
    (n / tiles)^2 run of the plain recipe.

    Each cell holds the exact mean of the continuous field over the cell (the
    Gaussian is separable; its cell means are differences of erf), so grids of
    any resolution hold finite-volume averages of one and the same field and a
    4x coarse graining of the n^2 state equals the (n/4)^2 state up to
    rounding.  Returns members first .. first + members - 1 of the seed's
    ensemble as ``[members][3][n][n]``."""
    edges = np.arange(n + 1, dtype=np.float64) / n
    specs = random_bump_specs(seed, (first + members) * tiles * tiles)[first * tiles * tiles:]
    inv = 1.0 / tiles
    kmax = 5 * tiles * tiles
    # bumps of every member padded to kmax with zero amplitude
    cx, cy = np.full((members, kmax), 0.5), np.full((members, kmax), 0.5)
    a, w = np.zeros((members, kmax)), np.full((members, kmax), inv)
    for b in range(members):
        k = 0
        for ty in range(tiles):
            for tx in range(tiles):
                spec = specs[(b * tiles + ty) * tiles + tx]
                m = len(spec.amps)
                cx[b, k:k + m] = (tx + spec.centres[:, 0]) * inv
                cy[b, k:k + m] = (ty + spec.centres[:, 1]) * inv
                a[b, k:k + m] = spec.amps
                w[b, k:k + m] = spec.widths * inv
                k += m
    ex = _gauss_cell_means(edges, cx.reshape(-1), w.reshape(-1)).reshape(members, kmax, n)
    ey = _gauss_cell_means(edges, cy.reshape(-1), w.reshape(-1)).reshape(members, kmax, n)
    q = np.zeros((members, 3, n, n))
    q[:, 0] = 1.0 + np.matmul((a[:, :, None] * ey).transpose(0, 2, 1), ex)   # h[b][j][i]
    return q


def swe_dam_break(nx: int, ny: int, h_left: float = 1.0, h_right: float = 0.35,
                  x0: float = 0.5) -> np.ndarray:
    """y-uniform dam break: h = h_left for x < x0, h_right otherwise, at rest.
    On the periodic square this holds two Riemann problems (at x0 and at 0)."""
    X, _ = _mesh(nx, ny)
    q = np.zeros((1, 3, ny, nx))
    q[0, 0] = np.where(X < x0, h_left, h_right)
    return q


def euler_sod(nx: int, ny: int, gamma: float = GAMMA_IDEAL, x0: float = 0.5,
              axis: str = "x") -> np.ndarray:
    """Sod shock tube, uniform across the other direction:
    (rho, u, p) = (1, 0, 1) left of x0 and (0.125, 0, 0.1) right of it."""
    X, Y = _mesh(nx, ny)
    s = X if axis == "x" else Y
    left = s < x0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    q = np.zeros((1, 4, ny, nx))
    q[0, 0] = rho
    q[0, 3] = p / (gamma - 1.0)
    return q


def swe_linear_wave(nx: int, ny: int, k: int = 1, eps: float = 1e-6,
                    depth: float = 1.0, g: float = G_GRAVITY) -> np.ndarray:
    """Small right-going gravity wave along x: h = H + eps sin(2 pi k x),
    hu = h * sqrt(g/H) * eps sin(2 pi k x) / H, hv = 0."""
    X, _ = _mesh(nx, ny)
    eta = eps * np.sin(2.0 * math.pi * k * X)
    h = depth + eta
    u = math.sqrt(g / depth) * eta / depth
    q = np.zeros((1, 3, ny, nx))
    q[0, 0] = h
    q[0, 1] = h * u
    return q


def euler_acoustic_wave(nx: int, ny: int, k: int = 1, eps: float = 1e-6,
                        rho0: float = 1.0, p0: float = 1.0,
                        gamma: float = GAMMA_IDEAL) -> np.ndarray:
    """Small right-going acoustic wave along x: rho = rho0 (1 + eps s),
    u = c eps s, p = p0 + rho0 c^2 eps s with s = sin(2 pi k x),
    c = sqrt(gamma p0 / rho0)."""
    X, _ = _mesh(nx, ny)
    s = np.sin(2.0 * math.pi * k * X)
    c = math.sqrt(gamma * p0 / rho0)
    rho = rho0 * (1.0 + eps * s)
    u = c * eps * s
    p = p0 + rho0 * c * c * eps * s
    q = np.zeros((1, 4, ny, nx))
    q[0, 0] = rho
    q[0, 1] = rho * u
    q[0, 3] = p / (gamma - 1.0) + 0.5 * rho * u * u
    return q


def random_smooth_swe(n: int, seed: int, members: int = 1, amp: float = 0.05,
                      vel: float = 0.05) -> np.ndarray:
    """Smooth random SWE states with non-zero velocity (few Fourier modes).
    Used where a test needs every term of the flux active."""
    rng = _rng(seed)
    X, Y = _mesh(n, n)
    q = np.zeros((members, 3, n, n))
    for b in range(members):
        fields = []
        for _ in range(3):
            f = np.zeros((n, n))
            for _m in range(4):
                kx, ky = rng.integers(-3, 4, size=2)
                ph = rng.uniform(0, 2 * math.pi)
                f += rng.normal() * np.cos(2 * math.pi * (kx * X + ky * Y) + ph)
            fields.append(f / 4.0)
        h = 1.0 + amp * fields[0]
        q[b, 0] = h
        q[b, 1] = h * vel * fields[1]
        q[b, 2] = h * vel * fields[2]
    return q


def perlin_bed(nx: int, ny: int, seed: int, cells: int = 6, octaves: int = 3,
               amp: float = 0.1) -> np.ndarray:
    """Water bed z [ny][nx] from 2D gradient (Perlin) noise, as in Section
    4.2's bathymetry test.

    Octave k has a lattice of ``cells * 2^k`` squares over the unit square,
    a seeded random unit gradient at each lattice node, and contributes the
    quintic-faded blend of the four corner ramps g . (p - node) at weight
    2^-k; the sum is shifted to mean 0 and scaled to max |z| = ``amp``.
    With the default depth h0 = 1 the water stays at least 0.9 deep."""
    rng = _rng(seed)
    X, Y = _mesh(nx, ny)
    z = np.zeros((ny, nx))
    for k in range(octaves):
        m = cells << k
        ang = rng.uniform(0.0, 2 * math.pi, size=(m + 1, m + 1))
        gx, gy = np.cos(ang), np.sin(ang)
        u, v = X * m, Y * m
        i0 = np.minimum(np.floor(u).astype(np.int64), m - 1)
        j0 = np.minimum(np.floor(v).astype(np.int64), m - 1)
        fu, fv = u - i0, v - j0

        def ramp(di, dj):
            return gx[j0 + dj, i0 + di] * (fu - di) + gy[j0 + dj, i0 + di] * (fv - dj)

        def fade(t):
            return t * t * t * (t * (6.0 * t - 15.0) + 10.0)

        wu, wv = fade(fu), fade(fv)
        bottom = ramp(0, 0) + wu * (ramp(1, 0) - ramp(0, 0))
        top = ramp(0, 1) + wu * (ramp(1, 1) - ramp(0, 1))
        z += (bottom + wv * (top - bottom)) / (1 << k)
    z -= z.mean()
    return amp * z / np.abs(z).max()


def swe_bump_over_bed(z: np.ndarray, amp: float = 0.1, width2: float = 0.005,
                      h0: float = 1.0) -> np.ndarray:
    """The Gaussian-hump surface of ``swe_gaussian_bump`` over the bed ``z``
    [ny][nx]: the free surface h + z is h0 plus the hump, at rest
    (Section 4.2 reuses the flat-bed initial condition).  Returns
    ``[1][3][ny][nx]``."""
    ny, nx = z.shape
    q = swe_gaussian_bump(nx, ny, amp, width2, h0)
    q[0, 0] -= z
    return q


def euler_four_quadrant(nx: int, ny: int, seed: int, split=(0.5, 0.5),
                        gamma: float = GAMMA_IDEAL) -> np.ndarray:
    """A 2D Riemann problem for Euler (Section 4.2's planar Euler test): four
    constant states in the quadrants around ``split``, drawn from the seed
    (rho in [0.5, 2], p in [0.3, 1.5], u and v in [-0.75, 0.75]).  The
    thesis runs one of Liska and Wendroff's configurations, whose states it
    does not print; these seeded states stand in for it.  Returns conserved
    variables ``[1][4][ny][nx]``; quadrant k = 0 (x, y >= split), 1 (x <
    split, y >= split), 2 (both below), 3 (x >= split, y < split)."""
    rng = _rng(seed)
    X, Y = _mesh(nx, ny)
    rho = rng.uniform(0.5, 2.0, 4)
    p = rng.uniform(0.3, 1.5, 4)
    u = rng.uniform(-0.75, 0.75, 4)
    v = rng.uniform(-0.75, 0.75, 4)
    east, north = X >= split[0], Y >= split[1]
    k = np.where(north, np.where(east, 0, 1), np.where(east, 3, 2))
    q = np.zeros((1, 4, ny, nx))
    q[0, 0] = rho[k]
    q[0, 1] = rho[k] * u[k]
    q[0, 2] = rho[k] * v[k]
    q[0, 3] = p[k] / (gamma - 1.0) + 0.5 * rho[k] * (u[k] ** 2 + v[k] ** 2)
    return q


@dataclasses.dataclass
class Request:
    """One solve request of the serving workload."""
    arrival_s: float
    eq: str           # "swe" or "euler"
    learned: bool
    n: int            # grid is n x n
    nsteps: int
    seed: int


def serving_requests(count: int, rate_per_s: float, seed: int = 42,
                     sizes=(64, 128, 256, 512, 1024, 2048),
                     horizon=(100, 5000)) -> list[Request]:
    """Poisson arrivals at ``rate_per_s``; grid side uniform over ``sizes``;
    horizon uniform integer in ``horizon``; 50 % learned SWE, 25 % plain SWE,
    25 % plain Euler (the learned variant exists for shallow water only)."""
    rng = _rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        kind = rng.uniform()
        if kind < 0.5:
            eq, learned = "swe", True
        elif kind < 0.75:
            eq, learned = "swe", False
        else:
            eq, learned = "euler", False
        out.append(Request(arrival_s=t, eq=eq, learned=learned,
                           n=int(rng.choice(np.asarray(sizes))),
                           nsteps=int(rng.integers(horizon[0], horizon[1] + 1)),
                           seed=int(seed * 1_000_003 + i)))
    return out


def request_initial_state(req: Request) -> np.ndarray:
    """Initial state of one request: random bumps (SWE) or KH (Euler)."""
    if req.eq == "swe":
        return swe_random_bumps(req.n, req.seed, 1)
    return euler_kelvin_helmholtz(req.n, req.n, seed=req.seed)


def as_f32_exact(q: np.ndarray) -> np.ndarray:
    """Round to FP32 and back: the exact values an FP32 GPU state starts from,
    which is what the oracle must be given for a like-for-like comparison."""
    return np.asarray(q, dtype=np.float32).astype(np.float64)


def sphere_bumps(centres: np.ndarray, seed: int, members: int = 1, depth: float = 1.2e-3,
                 amp: float = 2e-5, width2: float = 0.15, spin: float = 0.0) -> np.ndarray:
    """Shallow water on the unit sphere given its cell centres [3][ny][nx]
    (unit vectors; from the grid, e.g. ``sphere_get_cells``): depth plus
    three seeded Gaussian bumps amp exp(-|x - c_k|^2 / width2) at random unit
    centres c_k, and a seeded rigid rotation of angular speed ``spin``
    (momentum h (w x x), tangent to the sphere).  Section 4.3's test is the
    Rossby-Haurwitz wave of a published test suite; these states stand in
    for it.  Returns ``[members][4][ny][nx]`` (h, hu, hv, hw), float64."""
    rng = _rng(seed)
    x = np.asarray(centres, dtype=np.float64)
    _, ny, nx = x.shape
    q = np.zeros((members, 4, ny, nx))
    for b in range(members):
        h = np.full((ny, nx), depth)
        for _ in range(3):
            c = rng.normal(size=3)
            c /= np.linalg.norm(c)
            h += amp * np.exp(-((x - c[:, None, None]) ** 2).sum(0) / width2)
        w = rng.normal(size=3)
        w *= spin / np.linalg.norm(w)
        m = np.stack([w[1] * x[2] - w[2] * x[1], w[2] * x[0] - w[0] * x[2], w[0] * x[1] - w[1] * x[0]])
        q[b, 0] = h
        q[b, 1:] = m * h[None]
    return q
