"""Block domain decomposition of one large grid.

The explicit step reads a bounded stencil (2 cells for MUSCL-minmod, Eq.
2.18; 6 rows for the learned step, whose CNN reaches 4 cells beyond the 2 of
the reconstruction), so a periodic nx x ny grid splits into px x py blocks
that advance independently once a ring of their neighbours' cells is in place
before every Runge-Kutta stage.  A block is held as an ordinary library state
of (nx/px + 2 hx) x (ny/py + 2 hy) cells whose ring the library refreshes
(fv_halo_exchange within a process, fv_halo_pack / fv_halo_unpack between
processes); the next dt is the minimum over the blocks.  The interiors then
evolve exactly as the undecomposed grid.

* `Layout`: block geometry, periodic neighbours, split / join of whole-grid
  tensors (index plumbing only).
* `LocalDomain`: all blocks in one process on one GPU (the loopback case).
* `HaloComm`: the exchange of packed ring strips and the dt / diagnostics
  reductions between processes over torch.distributed, one block per rank,
  every wait bounded by a host-side limit (FV_ETIMEOUT when it runs out).
* `RankDomain`: one block per rank on its GPU, stepped with `HaloComm`.
* `allreduce_gradients`: the gradient reduction of data-parallel training.
"""
from __future__ import annotations

import ctypes
import dataclasses
import datetime

import numpy as np
import torch

from . import fv

SIDES = ("west", "east", "south", "north")
OPPOSITE = {0: 1, 1: 0, 2: 3, 3: 2}


@dataclasses.dataclass(frozen=True)
class Layout:
    """px x py blocks of an nx x ny periodic grid, each with a ring of hx
    columns (0 unless px > 1) and hy rows (0 unless py > 1)."""
    nx: int
    ny: int
    px: int
    py: int
    hx: int
    hy: int

    def __post_init__(self):
        if self.nx % self.px or self.ny % self.py:
            raise ValueError("the grid must split into equal blocks")
        if self.px > 1 and self.hx == 0 or self.py > 1 and self.hy == 0:
            raise ValueError("a split direction needs a ring")
        if 4 * self.hx > self.nx_ext or 4 * self.hy > self.ny_ext:
            raise ValueError("blocks too small for their rings")

    @staticmethod
    def make(nx: int, ny: int, px: int, py: int, halo: int) -> "Layout":
        """Rings of `halo` rows and of `halo` columns rounded up to a multiple
        of 4: the row-march stage kernel gives each thread 4 consecutive
        cells and evaluates their x faces partly as packed pairs, partly as a
        scalar, so a cell's results are the same bit for bit only where it
        keeps its column modulo 4 (the block width must then be a multiple
        of 4 too)."""
        hx = (halo + 3) // 4 * 4 if px > 1 else 0
        if px > 1 and (nx // px) % 4:
            raise ValueError("blocks split in x must be a multiple of 4 cells wide")
        return Layout(nx, ny, px, py, hx, halo if py > 1 else 0)

    @property
    def nxs(self) -> int:
        return self.nx // self.px

    @property
    def nys(self) -> int:
        return self.ny // self.py

    @property
    def nx_ext(self) -> int:
        return self.nxs + 2 * self.hx

    @property
    def ny_ext(self) -> int:
        return self.nys + 2 * self.hy

    @property
    def count(self) -> int:
        return self.px * self.py

    def block(self, k: int) -> tuple[int, int]:
        return k % self.px, k // self.px

    def neighbour(self, k: int, side: int) -> int:
        """Block on side 0 (west), 1 (east), 2 (south), 3 (north), periodic."""
        ix, iy = self.block(k)
        if side == 0:
            ix = (ix - 1) % self.px
        elif side == 1:
            ix = (ix + 1) % self.px
        elif side == 2:
            iy = (iy - 1) % self.py
        else:
            iy = (iy + 1) % self.py
        return iy * self.px + ix

    def extended(self, q: torch.Tensor, k: int) -> torch.Tensor:
        """Block k of a whole grid [..., ny, nx] with its ring (periodic)."""
        ix, iy = self.block(k)
        cols = (torch.arange(self.nx_ext, device=q.device) + ix * self.nxs - self.hx) % self.nx
        rows = (torch.arange(self.ny_ext, device=q.device) + iy * self.nys - self.hy) % self.ny
        return q.index_select(-1, cols).index_select(-2, rows).contiguous()

    def interior(self, qe: torch.Tensor) -> torch.Tensor:
        return qe[..., self.hy:self.hy + self.nys, self.hx:self.hx + self.nxs]

    def strip(self, qe: torch.Tensor, side: int, pack: bool) -> torch.Tensor:
        """View of an extended block [..., ny_ext, nx_ext]: the interior strip
        next to `side` that the neighbour there needs (pack) or the ring strip
        that the neighbour fills (unpack).  West/east strips span the interior
        rows, south/north strips the full width (the windows of
        fv_halo_pack / fv_halo_unpack)."""
        hx, hy, nxs, nys = self.hx, self.hy, self.nxs, self.nys
        if side < 2:
            x0 = (hx if side == 0 else nxs) if pack else (0 if side == 0 else nxs + hx)
            return qe[..., hy:hy + nys, x0:x0 + hx]
        y0 = (hy if side == 2 else nys) if pack else (0 if side == 2 else nys + hy)
        return qe[..., y0:y0 + hy, :]

    def split(self, q: torch.Tensor) -> list:
        return [self.extended(q, k) for k in range(self.count)]

    def join(self, blocks) -> torch.Tensor:
        b0 = blocks[0]
        out = torch.empty(b0.shape[:-2] + (self.ny, self.nx), dtype=b0.dtype, device=b0.device)
        for k, qe in enumerate(blocks):
            ix, iy = self.block(k)
            out[..., iy * self.nys:(iy + 1) * self.nys, ix * self.nxs:(ix + 1) * self.nxs] = self.interior(qe)
        return out


def _block_length(n_ext: int, n: int) -> float:
    """Domain length of an n_ext-cell block whose cells are those of an
    n-cell unit interval: the double nearest n_ext / n for which the library's
    own spacing length / n_ext is 1 / n bit for bit (the stage kernels then
    see the undecomposed grid's 1/dx)."""
    import math
    d = 1.0 / n
    cand = n_ext * d
    for _ in range(64):
        for c in (cand, math.nextafter(cand, math.inf), math.nextafter(cand, -math.inf)):
            if c / n_ext == d:
                return c
        cand = math.nextafter(cand, math.inf)
    raise ValueError(f"no block length gives spacing 1/{n} on {n_ext} cells")


def _init_block(q, eq, dt_mode, dt_fixed, cfl, layout):
    lx = _block_length(layout.nx_ext, layout.nx)
    ly = _block_length(layout.ny_ext, layout.ny)
    if eq == "swe":
        return fv.swe_init(q, cfl=cfl, dt_mode=dt_mode, dt_fixed=dt_fixed, lx=lx, ly=ly)
    return fv.euler_init(q, cfl=cfl, dt_mode=dt_mode, dt_fixed=dt_fixed, lx=lx, ly=ly)


def _global_hmin(q0: torch.Tensor, frac: float = 1e-3) -> np.ndarray:
    """The learned faces' positivity threshold of the whole grid: frac times
    each member's mean depth (what an undecomposed state fixes at its first
    learned step)."""
    return (frac * q0[:, 0].double().mean(dim=(1, 2))).cpu().numpy()


class LocalDomain:
    """All px x py blocks of one grid in this process, on the current GPU.
    q0: CUDA float32 [B][C][ny][nx]; the blocks share the caller's stream."""

    def __init__(self, q0: torch.Tensor, eq: str, px: int, py: int, halo: int = 2, dt_mode: str = "adaptive",
                 dt_fixed: float = 0.0, cfl: float = 0.5, learned: bool = False):
        B, C, ny, nx = q0.shape
        self.layout = Layout.make(nx, ny, px, py, halo)
        L = self.layout
        self.subs = [_init_block(qe, eq, dt_mode, dt_fixed, cfl, L) for qe in L.split(q0)]
        for s in self.subs:
            if L.hx or L.hy:
                fv.fv_set_halo(s, L.hx, L.hy)
        if learned:
            hmin = _global_hmin(q0)
            for s in self.subs:
                fv.fv_set_learned_hmin_values(s, hmin)
        self._arr = (ctypes.c_void_p * L.count)(*[s.handle.value for s in self.subs])
        fv.fv_reduce_dt(self._arr, L.count)

    def step(self, nsteps: int = 1, net=None) -> None:
        L = self.layout
        for _ in range(nsteps):
            fv.fv_halo_exchange(self._arr, L.px, L.py, 0)
            for s in self.subs:
                fv.fv_enqueue_stage(s, 1, net)
            fv.fv_halo_exchange(self._arr, L.px, L.py, 1)
            for s in self.subs:
                fv.fv_enqueue_stage(s, 2, net)
            fv.fv_reduce_dt(self._arr, L.count)

    def sync(self) -> None:
        for s in self.subs:
            fv.fv_sync(s)

    def state(self) -> torch.Tensor:
        return self.layout.join([fv.fv_get_state(s) for s in self.subs])

    def diagnostics(self) -> np.ndarray:
        """FP64 sums [B][C+1] of the whole grid: the blocks' interior sums added."""
        return sum(fv.fv_diagnostics(s) for s in self.subs)

    def time(self):
        return fv.fv_get_time(self.subs[0])


class HaloComm:
    """Ring strips and reductions between processes (one block per rank,
    rank = block index), over the default torch.distributed group: NCCL for
    CUDA tensors, gloo for host tensors.  Every wait is bounded by
    `timeout_s`; a peer that does not answer in time raises FvError with
    FV_ETIMEOUT (gloo then closes the connection, so the job stops there)."""

    def __init__(self, layout: Layout, rank: int, timeout_s: float = 30.0):
        import torch.distributed as dist
        if dist.get_world_size() != layout.count:
            raise ValueError("one block per rank")
        self.dist = dist
        self.L = layout
        self.rank = rank
        self.timeout = datetime.timedelta(seconds=timeout_s)

    def _wait(self, works, what):
        for w in works:
            try:
                w.wait(timeout=self.timeout)
            except RuntimeError as e:
                raise fv.FvError(fv.FV_ETIMEOUT, f"halo exchange ({what}): {e}") from e

    def exchange_phase(self, sides, send: dict, recv: dict) -> None:
        """Send send[side] to the neighbour on `side` and receive recv[side]
        from it, for the sides of one phase (west/east, then south/north).
        A strip sent west arrives as the neighbour's east ring (tag = the
        receiving side)."""
        works = []
        for side in sides:
            nb = self.L.neighbour(self.rank, side)
            if nb == self.rank:
                recv[side].copy_(send[OPPOSITE[side]])      # the block is its own neighbour
                continue
            works.append(self.dist.irecv(recv[side], src=nb, tag=side))
            works.append(self.dist.isend(send[side], dst=nb, tag=OPPOSITE[side]))
        self._wait(works, "/".join(SIDES[s] for s in sides))

    def _allreduce(self, t, op):
        w = self.dist.all_reduce(t, op=op, async_op=True)
        self._wait([w], "reduction")
        return t

    def min_dt(self, dt: np.ndarray) -> np.ndarray:
        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor(dt, dtype=torch.float64, device=dev)
        return self._allreduce(t, self.dist.ReduceOp.MIN).cpu().numpy()

    def sum(self, x: np.ndarray) -> np.ndarray:
        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor(x, dtype=torch.float64, device=dev)
        return self._allreduce(t, self.dist.ReduceOp.SUM).cpu().numpy()


class RankDomain:
    """One block of a grid decomposed over the ranks of torch.distributed
    (rank = block index, one GPU each): the block is a library state with a
    ring; before every stage its strips go to the neighbours through
    `HaloComm` (packed and unpacked by the library on the device), and the
    next dt is the minimum over the ranks."""

    def __init__(self, q_block: torch.Tensor, layout: Layout, comm: HaloComm, eq: str = "swe",
                 dt_mode: str = "adaptive", dt_fixed: float = 0.0, cfl: float = 0.5, hmin=None):
        self.L = layout
        self.comm = comm
        self.s = _init_block(q_block, eq, dt_mode, dt_fixed, cfl, layout)
        fv.fv_set_halo(self.s, layout.hx, layout.hy)
        if hmin is not None:
            fv.fv_set_learned_hmin_values(self.s, hmin)
        self._bufs = {}
        for side in range(4):
            if (side < 2 and layout.hx) or (side >= 2 and layout.hy):
                n = fv.fv_halo_strip_floats(self.s, side)
                self._bufs[side] = (torch.empty(n, device=q_block.device), torch.empty(n, device=q_block.device))
        self._min_dt()

    def _min_dt(self):
        _, dt, _ = fv.fv_get_time(self.s)
        fv.fv_set_dt(self.s, self.comm.min_dt(dt))

    def _refresh(self, buf: int):
        for phase in ((0, 1), (2, 3)):
            sides = [s for s in phase if s in self._bufs]
            if not sides:
                continue
            send = {s: self._bufs[s][0] for s in sides}
            recv = {s: self._bufs[s][1] for s in sides}
            for s in sides:
                fv.fv_halo_pack(self.s, buf, s, send[s])
            fv.fv_sync(self.s)
            self.comm.exchange_phase(sides, send, recv)
            for s in sides:
                fv.fv_halo_unpack(self.s, buf, s, recv[s])

    def step(self, nsteps: int = 1, net=None) -> None:
        for _ in range(nsteps):
            self._refresh(0)
            fv.fv_enqueue_stage(self.s, 1, net)
            self._refresh(1)
            fv.fv_enqueue_stage(self.s, 2, net)
            fv.fv_sync(self.s)
            self._min_dt()

    def interior(self) -> torch.Tensor:
        return self.L.interior(fv.fv_get_state(self.s))

    def diagnostics(self) -> np.ndarray:
        return self.comm.sum(fv.fv_diagnostics(self.s))


def allreduce_gradients(grad: torch.Tensor) -> torch.Tensor:
    """Data-parallel training: replace each rank's parameter gradient by the
    mean over the ranks (every rank then takes the same Adam step)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM)
        grad /= dist.get_world_size()
    return grad
