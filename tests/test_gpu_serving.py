"""The continuous-batching server: a request's result is the same alone and
in a mix of concurrent requests of different sizes, kinds and horizons;
admission respects the device-memory budget; an unstable request fails alone."""
import time

import numpy as np
import pytest
import torch

from paper_2602_08670_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv, train
    return fv, train


def _wait(fv, server, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            r = fv.poll(server, t)
            if r is not None:
                out[t] = r
        assert time.time() - t0 < timeout
        time.sleep(0.001)
    return out


def _mix():
    reqs = []
    for k, (eq, learned, n, steps) in enumerate([("swe", True, 64, 120), ("swe", False, 128, 200),
                                                 ("euler", False, 64, 150), ("swe", True, 128, 80),
                                                 ("swe", False, 64, 300), ("euler", False, 128, 60),
                                                 ("swe", True, 64, 33)]):
        r = W.Request(arrival_s=0.0, eq=eq, learned=learned, n=n, nsteps=steps, seed=100 + k)
        reqs.append((r, W.request_initial_state(r)[0].astype(np.float32)))
    return reqs


def test_results_same_alone_and_in_mix(mods):
    fv, TR = mods
    net, _ = TR.load_weights(TR_WEIGHTS(TR))
    reqs = _mix()
    server = fv.fv_server_create(8 << 30, 4, net)
    tickets = [fv.submit(server, q0, eq=r.eq, nsteps=r.nsteps, learned=r.learned,
                         cfl=0.4 if r.learned else 0.5) for r, q0 in reqs]
    mixed = _wait(fv, server, tickets)
    for (r, q0), t in zip(reqs, tickets):
        alone_srv = fv.fv_server_create(8 << 30, 1, net)
        ta = fv.submit(alone_srv, q0, eq=r.eq, nsteps=r.nsteps, learned=r.learned,
                       cfl=0.4 if r.learned else 0.5)
        alone = _wait(fv, alone_srv, [ta])[ta][0]
        assert np.array_equal(mixed[t][0], alone), (r.eq, r.learned, r.n)
        # and the same as a direct call of the library on the same state
        q = torch.tensor(q0[None]).cuda()
        st = fv.swe_init(q, cfl=0.4 if r.learned else 0.5) if r.eq == "swe" else fv.euler_init(q, cfl=0.5)
        fv.fv_rollout(st, r.nsteps, net=net if r.learned else None)
        assert np.array_equal(fv.fv_get_state(st).cpu().numpy()[0], alone)


def TR_WEIGHTS(TR):
    import os
    return os.path.join(os.path.dirname(TR.__file__), "weights", "swe64_from256.npz")


def test_admission_by_memory_budget(mods):
    fv, _ = mods
    reqs = [W.Request(0.0, "swe", False, 512, 400, 7 + k) for k in range(3)]
    one = 2 * 3 * 4 * 512 * 512 + (1 << 20)
    server = fv.fv_server_create(int(1.5 * one), 8)    # room for one 512^2 state at a time
    tickets = [fv.submit(server, W.request_initial_state(r)[0].astype(np.float32), nsteps=r.nsteps)
               for r in reqs]
    max_active = 0
    t0 = time.time()
    done = {}
    while len(done) < 3:
        a, p, used, _ = fv.fv_server_stats(server)
        max_active = max(max_active, a)
        assert used <= int(1.5 * one)
        for t in tickets:
            if t not in done:
                r = fv.poll(server, t)
                if r is not None:
                    done[t] = r
        assert time.time() - t0 < 120
    assert max_active == 1
    with pytest.raises(fv.FvError) as ei:
        fv.submit(server, np.ones((3, 1024, 1024), np.float32), nsteps=10)
    assert ei.value.code == fv.FV_EBUSY


def test_unstable_request_fails_alone(mods):
    fv, _ = mods
    server = fv.fv_server_create(1 << 30, 4)
    good = W.swe_random_bumps(64, 3, 1)[0].astype(np.float32)
    bad = good.copy()
    bad[0, 5, 5] = np.nan
    tg = fv.submit(server, good, nsteps=50)
    tb = fv.submit(server, bad, nsteps=50)
    t0 = time.time()
    res_good, err = None, None
    while res_good is None or err is None:
        if res_good is None:
            res_good = fv.poll(server, tg)
        if err is None:
            try:
                if fv.poll(server, tb) is not None:
                    err = "no error"
            except fv.FvError as e:
                err = e.code
        assert time.time() - t0 < 60
        time.sleep(0.001)
    assert err == fv.FV_EUNSTABLE
    assert np.isfinite(res_good[0]).all()


def test_unstable_learned_request_falls_back_to_plain_step(mods):
    fv, TR = mods
    rng = np.random.default_rng(0)
    wild = (rng.standard_normal(fv.FV_NET_PARAMS) * 0.5).astype(np.float32)   # far from stable
    net = fv.stencil_net_create(wild, [1.0, 0.0, 0.0], [0.2, 0.2, 0.2])
    server = fv.fv_server_create(1 << 30, 2, net)
    q0 = W.swe_random_bumps(64, 9, 1)[0].astype(np.float32)
    t = fv.submit(server, q0, nsteps=200, learned=True, cfl=0.4)
    res = _wait(fv, server, [t])[t][0]
    assert fv.fv_server_stats(server)[3] == 1
    q = torch.tensor(q0[None]).cuda()
    st = fv.swe_init(q, cfl=0.4)
    fv.fv_rollout(st, 200)
    assert np.array_equal(res, fv.fv_get_state(st).cpu().numpy()[0])
