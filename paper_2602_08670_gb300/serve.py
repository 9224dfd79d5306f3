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


def kernel_bound(requests, plain_rate: float, learned_rate: float) -> float:
    """Throughput the mix would reach if every request ran at its kernel's
    full-GPU rate one after another (plain requests at `plain_rate`, learned
    ones at `learned_rate`, in cell-updates/s): the work over the sum of the
    times."""
    t = sum(request_cell_updates(r) / (learned_rate if r.learned else plain_rate) for r in requests)
    return sum(request_cell_updates(r) for r in requests) / t


def sweep(server, base, fractions, seed: int = 42) -> dict:
    """Capacity (every request queued at t = 0), then Poisson arrivals at each
    fraction of it; initial states are built once, before any clock starts."""
    states = initial_states(base)
    closed = with_arrivals(base, 1e9, seed=seed)
    lat, span, fail = run_load(server, closed, states)
    cap = summarize(closed, lat, span, fail)
    out = {"capacity": cap, "load": []}
    for k, frac in enumerate(fractions):
        reqs = with_arrivals(base, frac * cap["requests_per_s"], seed=seed + 1 + k)
        lat, span, fail = run_load(server, reqs, states)
        d = summarize(reqs, lat, span, fail)
        d["rate_fraction_of_capacity"] = frac
        out["load"].append(d)
    return out


def main(argv=None):
    """The full serving workload: Poisson arrivals swept over fractions of the
    measured capacity, grids uniform over {64 .. 2048}^2, horizons uniform in
    [100, 5000] steps, 50 % learned SWE, 25 % plain SWE, 25 % plain Euler."""
    import argparse
    import json
    import os
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--fractions", default="0.1,0.25,0.5,0.75,0.9,1.0,1.2")
    ap.add_argument("--sizes", default="64,128,256,512,1024,2048")
    ap.add_argument("--horizon", default="100,5000")
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--slots", type=int, default=256)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    from . import train
    net, _ = train.load_weights(os.path.join(os.path.dirname(__file__), "weights", "swe64_from256.npz"))
    sizes = tuple(int(x) for x in a.sizes.split(","))
    horizon = tuple(int(x) for x in a.horizon.split(","))
    base = workloads.serving_requests(a.requests, 1.0, seed=42, sizes=sizes, horizon=horizon)
    server = fv.fv_server_create(int(a.budget_gb * (1 << 30)), a.slots, net)
    res = sweep(server, base, [float(x) for x in a.fractions.split(",")])
    res["workload"] = {"requests_per_rate": a.requests, "sizes": sizes, "horizon": horizon,
                       "mix": "50 % learned SWE, 25 % plain SWE, 25 % plain Euler", "seed": 42,
                       "budget_gb": a.budget_gb, "slots": a.slots}
    res["learned_fallbacks_to_plain"] = fv.fv_server_stats(server)[3]
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
