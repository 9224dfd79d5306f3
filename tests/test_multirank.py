"""Rank logic of multi-GPU runs, on CPU with gloo (world size 2).

Ranks share no data: each takes a shard of independent units, and the job's
throughput is all units over the slowest rank's time.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2602_08670_gb300 import ranks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_units, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = ranks.env()
        mine = ranks.shard(n_units, r, ws)
        # every rank sees every shard: they must tile [0, n_units) exactly
        gathered = [None] * ws
        dist.all_gather_object(gathered, (mine.start, mine.stop))
        # slowest rank decides the time; units add up
        secs = 1.0 + r            # rank r "took" 1 + r seconds
        rate, tmax = ranks.job_rate(len(mine), secs)
        ranks.barrier()
        with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
            json.dump({"ws": ws, "local": local, "gathered": gathered, "rate": rate,
                       "tmax": tmax, "max": ranks.max_over_ranks(10.0 * r),
                       "sum": ranks.sum_over_ranks(r + 1)}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_units", [7, 256, 1])
def test_gloo_two_ranks_shard_and_reduce(tmp_path, n_units):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), n_units, str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["ws"] == world and d["local"] == r
        spans = [tuple(x) for x in d["gathered"]]
        covered = [u for a, b in spans for u in range(a, b)]
        assert covered == list(range(n_units))          # disjoint, complete, ordered
        assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
        assert d["tmax"] == 2.0                          # slowest rank's time
        assert d["rate"] == pytest.approx(n_units / 2.0)
        assert d["max"] == 10.0 and d["sum"] == 3.0


def test_single_process_is_one_rank():
    assert ranks.shard(5, 0, 1) == range(0, 5)
    assert ranks.max_over_ranks(3.5) == 3.5
    rate, t = ranks.job_rate(10, 2.0)
    assert rate == 5.0 and t == 2.0
    with pytest.raises(ValueError):
        ranks.shard(5, 2, 2)
    with pytest.raises(ValueError):
        ranks.job_rate(1, 0.0)


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    """`bench.py --impl reference` under torchrun: rank 0 alone times the
    oracle and prints one JSON line; the other rank exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
