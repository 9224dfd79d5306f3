"""Load generator for the serving loop: Poisson arrivals of solve requests
(seeded request stream from ``workloads.serving_requests``) submitted to an
``fv_server`` in real time; reports throughput and latency percentiles."""
from __future__ import annotations

import time

import numpy as np

from . import fv, workloads


def request_cell_updates(req) -> float:
    return float(req.n) * req.n * req.nsteps


def initial_states(requests) -> list:
    """Host FP32 initial state [C][n][n] of every request, built before the
    load starts so that generating inputs is not part of the latencies."""
    return [np.ascontiguousarray(workloads.request_initial_state(r)[0].astype(np.float32))
            for r in requests]


def run_load(server, requests, states=None, learned_cfl: float = 0.4, plain_cfl: float = 0.5,
             poll_interval: float = 0.0005):
    """Submit each request at its arrival time (its initial state from
    ``states``, else built before the clock starts), poll until all are
    done.  Returns (latencies [s], makespan [s], failures)."""
    if states is None:
        states = initial_states(requests)
    t0 = time.perf_counter()
    pending = {}
    lat = []
    failures = 0
    i = 0
    while i < len(requests) or pending:
        now = time.perf_counter() - t0
        while i < len(requests) and requests[i].arrival_s <= now:
            r = requests[i]
            t = fv.submit(server, states[i], eq=r.eq, nsteps=r.nsteps, learned=r.learned,
                          cfl=learned_cfl if r.learned else plain_cfl)
            pending[t] = r
            i += 1
        for t in list(pending):
            try:
                res = fv.poll(server, t)
            except fv.FvError:
                failures += 1
                del pending[t]
                continue
            if res is not None:
                lat.append(res[1])
                del pending[t]
        time.sleep(poll_interval)
    return np.asarray(lat), time.perf_counter() - t0, failures


def summarize(requests, lat, makespan, failures) -> dict:
    work = sum(request_cell_updates(r) for r in requests)
    return {"requests": len(requests), "failures": failures,
            "throughput_cell_updates_per_s": work / makespan,
            "requests_per_s": len(requests) / makespan,
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_latency_s": float(lat.mean()) if len(lat) else None}


def with_arrivals(requests, rate_per_s: float, seed: int):
    """Same requests, Poisson arrival times at rate_per_s."""
    rng = np.random.Generator(np.random.Philox(seed + 7))
    t = 0.0
    out = []
    for r in requests:
        t += rng.exponential(1.0 / rate_per_s)
        out.append(workloads.Request(arrival_s=t, eq=r.eq, learned=r.learned, n=r.n,
                                     nsteps=r.nsteps, seed=r.seed))
    return out
