"""Block domain decomposition on the CPU: the layout, the stage-by-stage
protocol with the FP64 oracle stepping every block on its extended grid
(bitwise equal to the undecomposed oracle run), halo strips exchanged between
gloo ranks (world size 2), a late peer that runs out the host-side time limit,
and the gradient all-reduce of data-parallel training."""
import datetime
import json
import os
import socket
import time

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import fv as ofv
from paper_2602_08670_gb300 import decomp
from paper_2602_08670_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _swe(n, seed):
    return torch.tensor(W.random_smooth_swe(n, seed=seed, members=2, amp=0.1, vel=0.3))


def _euler(n, seed):
    return torch.tensor(np.concatenate([W.euler_kelvin_helmholtz(n, n, seed=seed + k) for k in range(2)]))


def test_layout_split_join_and_neighbours():
    q = torch.arange(2 * 3 * 12 * 16, dtype=torch.float64).reshape(2, 3, 12, 16)
    L = decomp.Layout.make(32, 12, 2, 3, 2)
    assert L.hx == 4 and L.hy == 2           # x rings keep columns modulo 4
    blocks = L.split(q := torch.arange(2 * 3 * 12 * 32, dtype=torch.float64).reshape(2, 3, 12, 32))
    assert len(blocks) == 6 and blocks[0].shape == (2, 3, 8, 24)
    assert torch.equal(L.join(blocks), q)
    # the ring of block 0 (ix = iy = 0) wraps to the last columns / rows
    assert torch.equal(blocks[0][..., 2:6, 0:4], q[..., 0:4, 28:32])
    assert torch.equal(blocks[0][..., 0:2, 4:20], q[..., 10:12, 0:16])
    assert torch.equal(blocks[0][..., 0:2, 0:4], q[..., 10:12, 28:32])      # corner
    assert L.neighbour(0, 0) == 1 and L.neighbour(0, 1) == 1
    assert L.neighbour(0, 2) == 4 and L.neighbour(0, 3) == 2
    # a strip packed on one side is the neighbour's ring on the opposite side
    for k in range(L.count):
        for side in range(4):
            nb = L.neighbour(k, side)
            assert torch.equal(L.strip(blocks[k], side, True), L.strip(blocks[nb], decomp.OPPOSITE[side], False)) \
                or side >= 2      # y strips span the rings, which hold x neighbours' cells
    one = decomp.Layout.make(16, 12, 1, 2, 2)
    assert one.hx == 0 and one.hy == 2 and one.nx_ext == 16 and one.ny_ext == 10
    with pytest.raises(ValueError):
        decomp.Layout(16, 12, 2, 1, 0, 0)     # split without a ring
    with pytest.raises(ValueError):
        decomp.Layout.make(20, 12, 2, 1, 2)   # 10-cell blocks would shift columns modulo 4


def _oracle_step_blocks(blocks, L, eq, dx, dy, cfl, refresh):
    """One SSP-RK2 step of every block on its extended grid (Eq. 2.19 in the
    oracle's own arithmetic), dt from the largest interior Courant rate."""
    rate = torch.stack([ofv.max_courant_rate(L.interior(b), eq, dx, dy) for b in blocks]).amax(dim=0)
    dt = (cfl / rate).view(-1, 1, 1, 1)
    q1 = [b + dt * ofv.rhs(b, eq, dx, dy) for b in blocks]
    q1 = refresh(q1)
    return [0.5 * b + 0.5 * c + 0.5 * dt * ofv.rhs(c, eq, dx, dy) for b, c in zip(blocks, q1)], dt


@pytest.mark.parametrize("eq,px,py", [("swe", 2, 2), ("swe", 4, 1), ("euler", 1, 4), ("euler", 2, 2)])
def test_oracle_blocks_equal_the_whole_grid(eq, px, py):
    n = 32
    q0 = _swe(n, 3) if eq == "swe" else _euler(n, 3)
    steps = 6
    ref, t_ref, _, _ = ofv.run(q0, eq, steps, cfl=0.5)
    L = decomp.Layout.make(n, n, px, py, 2)

    def refresh(blocks):
        return L.split(L.join(blocks))

    blocks = L.split(q0)
    t = 0
    for _ in range(steps):
        blocks, dt = _oracle_step_blocks(blocks, L, eq, 1 / n, 1 / n, 0.5, refresh)
        blocks = refresh(blocks)
        t = t + dt.view(-1)
    assert torch.equal(L.join(blocks), ref)
    assert torch.equal(t, t_ref)
    # diagnostics of the whole grid = sums of the blocks' interior diagnostics
    d = sum(ofv.diagnostics(L.interior(b), eq) for b in blocks) * 1.0
    # (diagnostics() scales by the cell area of its argument's own shape)
    scale = (1 / (L.nxs * L.nys)) / (1 / (n * n))
    assert torch.allclose(d / scale, ofv.diagnostics(ref, eq), rtol=1e-13, atol=1e-14)


def _rank_worker(rank, world, port, eq, px, py, out_dir, late):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    n, steps = 32, 4
    q0 = _swe(n, 5) if eq == "swe" else _euler(n, 5)
    L = decomp.Layout.make(n, n, px, py, 2)
    comm = decomp.HaloComm(L, rank, timeout_s=1.5)
    mine = L.extended(q0, rank)
    status = 0
    try:
        if late and rank == 1:
            time.sleep(4.0)            # a peer that misses the exchange's time limit

        def refresh(blocks):
            (b,) = blocks
            for phase in ((0, 1), (2, 3)):
                sides = [s for s in phase if (L.hx if s < 2 else L.hy)]
                if not sides:
                    continue
                send = {s: L.strip(b, s, True).contiguous() for s in sides}
                recv = {s: torch.empty_like(L.strip(b, s, False)) for s in sides}
                comm.exchange_phase(sides, send, recv)
                for s in sides:
                    L.strip(b, s, False).copy_(recv[s])
            return [b]

        blocks = refresh([mine])
        for _ in range(steps):
            rate = ofv.max_courant_rate(L.interior(blocks[0]), eq, 1 / n, 1 / n)
            rate = -torch.tensor(comm.min_dt(-rate.numpy()))        # max over ranks
            dt = (0.5 / rate).view(-1, 1, 1, 1)
            b = blocks[0]
            q1 = refresh([b + dt * ofv.rhs(b, eq, 1 / n, 1 / n)])[0]
            blocks = refresh([0.5 * b + 0.5 * q1 + 0.5 * dt * ofv.rhs(q1, eq, 1 / n, 1 / n)])
        gathered = [None] * world
        dist.all_gather_object(gathered, blocks[0].numpy())
        diag = comm.sum(ofv.diagnostics(L.interior(blocks[0]), eq).numpy())
        if rank == 0:
            full = L.join([torch.tensor(g) for g in gathered])
            ref, _, _, _ = ofv.run(q0, eq, steps, cfl=0.5)
            res = {"equal": bool(torch.equal(full, ref)), "diag": diag.tolist(),
                   "maxdiff": float((full - ref).abs().max()),
                   "diag_ref": (ofv.diagnostics(ref, eq) * (n * n) / (L.nxs * L.nys)).numpy().tolist()}
            with open(os.path.join(out_dir, "res.json"), "w") as f:
                json.dump(res, f)
    except Exception as e:          # noqa: BLE001 - the status is the test's subject
        status = getattr(e, "code", -99)
        t_fail = time.time()
        with open(os.path.join(out_dir, f"status{rank}.json"), "w") as f:
            json.dump({"status": status, "msg": str(e)[:300], "t": t_fail}, f)
        return                      # the connection is gone: leave without collectives
    dist.destroy_process_group()


@pytest.mark.parametrize("eq,px,py", [("swe", 2, 1), ("euler", 1, 2)])
def test_gloo_ranks_exchange_halos(tmp_path, eq, px, py):
    mp.start_processes(_rank_worker, args=(2, _free_port(), eq, px, py, str(tmp_path), False),
                       nprocs=2, join=True, start_method="spawn")
    res = json.load(open(tmp_path / "res.json"))
    assert res["equal"]                    # bitwise the undecomposed oracle run
    assert np.allclose(res["diag"], res["diag_ref"], rtol=1e-13, atol=1e-14)


def test_gloo_late_peer_times_out(tmp_path):
    t0 = time.time()
    mp.start_processes(_rank_worker, args=(2, _free_port(), "swe", 2, 1, str(tmp_path), True),
                       nprocs=2, join=True, start_method="spawn")
    st0 = json.load(open(tmp_path / "status0.json"))
    assert st0["status"] == -4, st0        # FV_ETIMEOUT on the rank that waited
    assert st0["t"] - t0 < 60
    st1 = json.load(open(tmp_path / "status1.json"))
    assert st1["status"] != 0              # the late rank finds the exchange closed


def _grad_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = torch.full((29796,), float(rank + 1))
    g[0] = 10.0 * rank
    decomp.allreduce_gradients(g)
    if rank == 0:
        np.save(os.path.join(out_dir, "g.npy"), g.numpy())
    dist.destroy_process_group()


def test_gloo_gradient_allreduce_is_the_mean(tmp_path):
    mp.start_processes(_grad_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    g = np.load(tmp_path / "g.npy")
    assert g[0] == 5.0 and np.all(g[1:] == 1.5)
