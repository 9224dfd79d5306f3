"""Training and evaluation of the learned solvers (GPU, via libfv): the
stencil network (Section 2.5.3, fourth approach) and the face-state network
(third approach).

Data (Section 2.5.1 / 5.4 recipe, on this build's synthetic workload): the
plain FP32 GPU solver runs seeded multi-bump shallow-water states at a fine
resolution (256^2) with a fixed dt; every `factor` fine steps the state is
block-averaged `factor` x `factor` down to the coarse grid (64^2), so one
coarse step = `factor` fine steps.  Training windows are (q_k, q_{k+1} ..
q_{k+T}) from those sequences; the loss is Eq. 2.28 on a T-step learned
rollout at the coarse resolution, minimised with Adam.  All numerical work
(solver, coarse graining, CNN forward / backward, loss, Adam) runs in the CUDA
library; this module samples windows and calls it.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np
import torch

from . import fv, workloads

G = 9.81
LAYERS = [(32, 3), (32, 32), (32, 32), (36, 32)]
FACE_LAYERS = [(32, 3), (32, 32), (32, 32), (12, 32)]


@dataclasses.dataclass
class Dataset:
    coarse: torch.Tensor      # [S][B][3][nc][nc] (CUDA)
    dt_coarse: float
    dt_fine: float
    n_fine: int
    factor: int
    seed: int

    @property
    def n_coarse(self) -> int:
        return self.n_fine // self.factor


def stable_fine_dt(n_fine: int, seed: int, members: int, cfl: float = 0.5, safety: float = 0.8) -> float:
    """Fixed fine dt: the adaptive (CFL) dt the library computes for the
    initial states, minimum over members, times a safety factor."""
    q0 = torch.tensor(workloads.swe_random_bumps(n_fine, seed, members), dtype=torch.float32).cuda()
    st = fv.swe_init(q0, cfl=cfl)
    _, ndt, _ = fv.fv_get_time(st)
    return float(safety * ndt.min())


def generate(n_fine: int = 256, factor: int = 4, members: int = 64, seed: int = 0,
             coarse_steps: int = 128, dt_fine: float | None = None) -> Dataset:
    """Fine plain-solver trajectories coarse-grained to n_fine / factor."""
    if dt_fine is None:
        dt_fine = stable_fine_dt(n_fine, seed, members)
    q0 = torch.tensor(workloads.swe_random_bumps(n_fine, seed, members), dtype=torch.float32).cuda()
    st = fv.swe_init(q0, dt_mode="fixed", dt_fixed=dt_fine)
    nc = n_fine // factor
    coarse = torch.empty((coarse_steps + 1, members, 3, nc, nc), dtype=torch.float32, device="cuda")
    coarse[0] = fv.fv_coarsen(q0, factor)
    buf = torch.empty_like(q0)
    for k in range(1, coarse_steps + 1):
        fv.fv_rollout(st, factor)
        fv.fv_get_state(st, out=buf)
        coarse[k] = fv.fv_coarsen(buf, factor)
    return Dataset(coarse, dt_fine * factor, dt_fine, n_fine, factor, seed)


def init_params(seed: int, zero_last: bool = True, kind: str = "stencil", depth: float = 1.0) -> np.ndarray:
    """He-normal weights, small biases.  Stencil network: a zero last layer
    makes it start as the first-order scheme (the paper's initialisation).
    Face-state network (no initialisation is given for it): a zero last
    layer with depth biases softplus^-1(depth) starts every side at the
    resting depth with zero momentum."""
    g = torch.Generator().manual_seed(seed)
    layers = FACE_LAYERS if kind == "face" else LAYERS
    parts = []
    for layer, (co, ci) in enumerate(layers):
        w = torch.randn(co, ci, 3, 3, generator=g) * math.sqrt(2.0 / (9 * ci))
        b = torch.randn(co, generator=g) * 0.01
        if layer == 3 and zero_last:
            w.zero_()
            b.zero_()
            if kind == "face":
                b[0::3] = math.log(math.expm1(depth))
        parts += [w.reshape(-1), b]
    return torch.cat(parts).numpy().astype(np.float32)


def data_stats(ds: Dataset):
    """Per-variable mean and standard deviation of the coarse training states
    (the loss scale of Eq. 2.28)."""
    x = ds.coarse.transpose(0, 2).reshape(3, -1).double()
    mean = x.mean(dim=1).cpu().numpy()
    std = np.maximum(x.std(dim=1).cpu().numpy(), 1e-6)
    return mean.astype(np.float32), std.astype(np.float32)


def input_scale(ds: Dataset):
    """Per-variable mean and largest absolute deviation from it: the CNN input
    normalisation x = (q - mean) / scale maps the training states into
    [-1, 1].  (The standard deviation is dominated by the flat background, so
    dividing by it puts the bumps at 15-20 and makes every Adam step a large
    change of the stencils.)"""
    x = ds.coarse.transpose(0, 2).reshape(3, -1).double()
    mean = x.mean(dim=1)
    dev = (x - mean[:, None]).abs().amax(dim=1).cpu().numpy()
    return mean.cpu().numpy().astype(np.float32), np.maximum(dev, 1e-6).astype(np.float32)


@dataclasses.dataclass
class TrainResult:
    net: object
    losses: list
    seconds: float
    iters: int
    rejected: int
    lr: float


def train(ds: Dataset, iters: int = 500, batch: int = 64, T: int = 8, lr: float = 3e-4,
          seed: int = 0, params=None, log_every: int = 0, net=None, kind: str = "stencil",
          pushforward: int = 0) -> TrainResult:
    """Adam on the rollout loss.  An update after which a training rollout
    leaves the physical states (the library reports FV_EUNSTABLE) is undone
    and the learning rate halved.

    pushforward = K > 0: before each batch the current network advances the
    window starts by k ~ U{0..K} learned steps without a tape, and the loss
    is taken on the T taped steps that follow, against the reference at the
    matching times; the network learns to correct the states of its own long
    rollouts without differentiating through them.  A batch whose untaped
    steps leave the physical states is skipped (learning rate unchanged)."""
    mean, std = data_stats(ds)
    if net is None:
        in_mean, in_scale = input_scale(ds)
        if kind == "face":
            p0 = init_params(seed, kind="face", depth=float(mean[0])) if params is None else params
            net = fv.face_net_create(p0, in_mean, in_scale)
        else:
            net = fv.stencil_net_create(init_params(seed) if params is None else params, in_mean, in_scale)
    S, B = ds.coarse.shape[:2]
    nc = ds.n_coarse
    tape = fv.fv_tape_create(net, batch, nc, nc, T, ds.dt_coarse)
    dparams = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    prev = torch.empty_like(dparams)
    fv.stencil_net_get_params(net, out=prev)
    rng = np.random.Generator(np.random.Philox(seed))
    scale = std
    losses = []
    rejected = 0
    step = 0
    pre = None
    if pushforward:
        pre = fv.swe_init(ds.coarse[0, :batch].contiguous(), dt_mode="fixed", dt_fixed=ds.dt_coarse)
    t0 = time.perf_counter()
    for it in range(iters):
        traj = torch.tensor(rng.integers(0, B, size=batch), device="cuda")
        k_pre = int(rng.integers(0, pushforward + 1)) if pushforward else 0
        start = torch.tensor(rng.integers(0, S - T - k_pre, size=batch), device="cuda")
        q0 = ds.coarse[start, traj].contiguous()
        targets = torch.stack([ds.coarse[start + k_pre + k, traj] for k in range(1, T + 1)]).contiguous()
        if k_pre:
            fv.fv_set_state(pre, q0)
            try:
                fv.fv_rollout(pre, k_pre, net=net)
                q0 = fv.fv_get_state(pre)
            except fv.FvError as e:
                if e.code != fv.FV_EUNSTABLE:
                    raise
                # a fresh state: the health word of this one stays set
                pre = fv.swe_init(ds.coarse[0, :batch].contiguous(), dt_mode="fixed", dt_fixed=ds.dt_coarse)
                rejected += 1
                continue
        try:
            fv.fv_tape_forward(tape, q0, want_snaps=False)
        except fv.FvError as e:
            if e.code != fv.FV_EUNSTABLE:
                raise
            fv.stencil_net_set_params(net, prev)
            if not pushforward:
                lr *= 0.5
            rejected += 1
            continue
        losses.append(fv.fv_tape_loss(tape, targets, scale))
        dparams.zero_()
        fv.fv_tape_backward(tape, dparams)
        fv.stencil_net_get_params(net, out=prev)
        step += 1
        fv.stencil_net_adam_step(net, dparams, step, lr)
        if log_every and (it + 1) % log_every == 0:
            print(f"iter {it + 1}: loss {np.mean(losses[-log_every:]):.5g}", flush=True)
    torch.cuda.synchronize()
    return TrainResult(net, losses, time.perf_counter() - t0, iters, rejected, lr)


def rel_l2(a: torch.Tensor, ref: torch.Tensor) -> list:
    """Per-variable relative L2 error over all members and cells."""
    return [float((a[:, c] - ref[:, c]).norm() / ref[:, c].norm()) for c in range(a.shape[1])]


def state_error(a: torch.Tensor, ref: torch.Tensor, scale) -> float:
    """RMS of the scaled state difference (the per-variable normalisation of
    the training loss), over all members, cells and variables."""
    s = torch.as_tensor(np.asarray(scale), dtype=torch.float64, device=a.device).view(1, -1, 1, 1)
    d = (a.double() - ref.double()) / s
    return float(torch.sqrt((d * d).mean()))


def rollout_coarse(q0: torch.Tensor, dt: float, nsteps: int, net=None) -> torch.Tensor:
    st = fv.swe_init(q0.contiguous(), dt_mode="fixed", dt_fixed=dt)
    fv.fv_rollout(st, nsteps, net=net)
    return fv.fv_get_state(st)


def evaluate(net, ds: Dataset, nsteps: int, scale) -> dict:
    """Learned and plain coarse solvers from ds.coarse[0], nsteps coarse steps,
    against the coarse-grained fine reference ds.coarse[nsteps]."""
    q0 = ds.coarse[0]
    ref = ds.coarse[nsteps]
    ql = rollout_coarse(q0, ds.dt_coarse, nsteps, net)
    qp = rollout_coarse(q0, ds.dt_coarse, nsteps, None)
    return {"learned": state_error(ql, ref, scale), "plain": state_error(qp, ref, scale),
            "learned_rel_l2": rel_l2(ql, ref), "plain_rel_l2": rel_l2(qp, ref)}


def plain_error_at(n: int, ds: Dataset, nsteps: int, scale) -> float:
    """Error against the same reference of the plain solver run at n^2 (from
    the same continuous initial field) and coarse-grained to the coarse grid."""
    factor = n // ds.n_coarse
    assert factor * ds.n_coarse == n
    members = ds.coarse.shape[1]
    q0 = torch.tensor(workloads.swe_random_bumps(n, ds.seed, members), dtype=torch.float32).cuda()
    ratio = ds.n_fine / n
    dt = ds.dt_fine * ratio
    steps = int(round(nsteps * ds.factor / ratio))
    q = rollout_coarse(q0, dt, steps)
    return state_error(fv.fv_coarsen(q, factor), ds.coarse[nsteps], scale)


def _tiled_state(n: int, seed: int, members: int, tiles: int, chunk: int = 16) -> torch.Tensor:
    """swe_random_bumps_tiled on the device, generated in member chunks."""
    out = torch.empty((members, 3, n, n), dtype=torch.float32, device="cuda")
    for b0 in range(0, members, chunk):
        m = min(chunk, members - b0)
        q = workloads.swe_random_bumps_tiled(n, seed, m, tiles, first=b0)
        out[b0:b0 + m] = torch.from_numpy(q.astype(np.float32))
    return out


def remap_mean(q: torch.Tensor, n: int) -> torch.Tensor:
    """Cell averages on the n x n grid of a piecewise-constant [B][C][N][N]
    field (N >= n): duplicate every cell k x k times so that n divides N k,
    then take the block means (the coarse-graining kernel)."""
    N = q.shape[-1]
    if N == n:
        return q
    k = n // math.gcd(N, n)
    if k > 1:
        q = q.repeat_interleave(k, dim=-1).repeat_interleave(k, dim=-2)
    return fv.fv_coarsen(q.contiguous(), N * k // n)


class _ErrAcc:
    """Accumulates, over member chunks, the error measures of a coarse state
    against the reference: relative L2 per variable, Section 3's mean
    relative depth error (E1), and the RMS of the per-variable scaled
    difference (the normalisation of the Eq. 2.28 loss)."""

    def __init__(self, scale):
        self.s = torch.as_tensor(np.asarray(scale), dtype=torch.float64, device="cuda").view(1, -1, 1, 1)
        self.d2 = torch.zeros(3, dtype=torch.float64, device="cuda")
        self.r2 = torch.zeros(3, dtype=torch.float64, device="cuda")
        self.e1 = torch.zeros((), dtype=torch.float64, device="cuda")
        self.sc = torch.zeros((), dtype=torch.float64, device="cuda")
        self.cells = 0

    def add(self, a: torch.Tensor, ref: torch.Tensor) -> None:
        a, ref = a.double(), ref.double()
        d = a - ref
        self.d2 += (d * d).sum(dim=(0, 2, 3))
        self.r2 += (ref * ref).sum(dim=(0, 2, 3))
        self.e1 += (d[:, 0].abs() / ref[:, 0]).sum()
        self.sc += ((d / self.s) ** 2).sum()
        self.cells += ref[:, 0].numel()

    def result(self) -> dict:
        rel = (self.d2 / self.r2).sqrt().tolist()
        return {"scaled_rms": float((self.sc / (3 * self.cells)).sqrt()), "rel_l2": rel,
                "e1_mean_rel_h": float(self.e1 / self.cells)}


def _interp_resolution(errs: dict, err: float):
    """Resolution at which the plain solver's error equals err: log-log
    interpolation between the bracketing resolutions (None outside)."""
    ns = sorted(errs)
    for a, b in zip(ns, ns[1:]):
        ea, eb = errs[a], errs[b]
        if ea >= err >= eb and ea > eb:
            t = (math.log(ea) - math.log(err)) / (math.log(ea) - math.log(eb))
            return math.exp(math.log(a) + t * (math.log(b) - math.log(a)))
    return None


def _timed_rollout(q0: torch.Tensor, dt: float, segments, net=None, keep=True, stream=None,
                   flags=None, seg_ms=None):
    """Fixed-dt rollout of q0 in consecutive segments of steps; returns (the
    state after each segment (device copies) or None, device milliseconds of
    the steps (CUDA events on the state's stream), members flagged unstable).
    `flags`, if a list, receives each member's health word after every
    segment, `seg_ms` the device milliseconds of every segment."""
    bs = stream or torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(bs):
        st = fv.swe_init(q0, dt_mode="fixed", dt_fixed=dt)
    out, ms = [], 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def tolerate_unstable(call, *a):
        # a member that left the physical states is reported (health word),
        # and its NaNs show in the errors; the others carry on
        try:
            return call(*a)
        except fv.FvError as e:
            if e.code != fv.FV_EUNSTABLE:
                raise
            return a[-1] if len(a) > 1 else None

    for k in segments:
        torch.cuda.synchronize()
        e0.record(bs)
        fv.fv_enqueue_steps(st, k, net=net)
        e1.record(bs)
        tolerate_unstable(fv.fv_sync, st)
        ms += e0.elapsed_time(e1)
        if seg_ms is not None:
            seg_ms.append(e0.elapsed_time(e1))
        if flags is not None:
            flags.append(fv.fv_health(st).copy())
        if keep:
            buf = torch.empty(tuple(q0.shape), dtype=torch.float32, device="cuda")
            out.append(tolerate_unstable(lambda s_, b_: fv.fv_get_state(s_, out=b_), st, buf))
    bad = int((fv.fv_health(st) != 0).sum())
    del st
    return (out if keep else None), ms, bad


def matched_accuracy(nets: dict, dt_coarse64: float, scale, n: int = 256, tiles: int = 4,
                     members: int = 256, seed: int = 3, horizons=(64, 256, 1000, 2000),
                     plain_factors=(1.0, 1.5, 2.0, 3.0), headline: int | None = None) -> dict:
    """Learned versus plain at matched accuracy on one configuration (Section
    5.4's comparison; Eq. 2.28's error normalisation).

    Workload: `members` states of swe_random_bumps_tiled(n, seed, ., tiles),
    the training recipe with features scaled to the n^2 grid, so that a
    network trained on the 64^2 coarse graining of 256^2 runs applies with
    the coarse step dt_coarse64 * 64 / n.  Reference: the plain solver at
    (4 n)^2 with a 4x smaller step, coarse-grained 4x (the training data's
    coarse graining).  Each learned network runs once, timed (CUDA events),
    and its state at every horizon is compared with the reference; the plain
    solver runs at N = f n for f in plain_factors (steps and dt scaled by f),
    remapped to n^2 by cell averages.  N_eq interpolates, in log-log, the
    plain error over N to the learned error; the plain solver is then timed
    at N_eq itself (rounded to a multiple of 4).  The accuracy-matched rate
    is the plain work at N_eq (N_eq^2 cells x K N_eq / n steps per member)
    over the learned run's time: learned rate x (N_eq / n)^3.

    The learned solver runs with the plain step as its fallback: a member the
    library flags as having left the physical states (health word) is run
    again from its initial state by the plain solver at n^2, whose states
    replace the learned ones from the first horizon at which the member was
    flagged, and whose device time is added to the learned time (the same
    rule as the server's restart of an unstable learned request)."""
    assert all(k % 2 == 0 for k in horizons)
    headline = headline or horizons[-1]
    dt = dt_coarse64 * 64.0 / n
    segs = [horizons[0]] + [b - a for a, b in zip(horizons, horizons[1:])]
    out = {"workload": f"{members} members x {n}^2 SWE, random bumps scaled to the grid ({tiles}x{tiles} "
                       f"tiles of the 64^2 training recipe, seed {seed}), fixed dt {dt:.4g}",
           "reference": f"plain solver at {4 * n}^2, dt/4, coarse-grained 4x",
           "horizons": list(horizons), "headline_horizon": headline}
    bs = torch.cuda.Stream()
    # reference at 4n
    qf = _tiled_state(4 * n, seed, members, tiles)
    refs, ref_ms, _ = _timed_rollout(qf, dt / 4, [4 * k for k in segs], stream=bs)
    del qf
    refs = [fv.fv_coarsen(r, 4) for r in refs]
    torch.cuda.empty_cache()
    q0 = _tiled_state(n, seed, members, tiles)
    # plain solver at N = f n
    plain = {}
    for f in plain_factors:
        N = int(round(f * n))
        qN = q0 if N == n else _tiled_state(N, seed, members, tiles)
        states, ms, bad = _timed_rollout(qN, dt * n / N, [int(round(k * f)) for k in segs], stream=bs)
        errs = []
        for st, ref in zip(states, refs):
            acc = _ErrAcc(scale)
            for b0 in range(0, members, 16):
                acc.add(remap_mean(st[b0:b0 + 16], n), ref[b0:b0 + 16])
            errs.append(acc.result())
        steps = int(round(horizons[-1] * f))
        plain[N] = {"errors": errs, "cell_updates_per_s": members * N * N * steps / (ms * 1e-3),
                    "unstable_members": bad}
        del states
        torch.cuda.empty_cache()
    out["plain"] = {str(N): v for N, v in plain.items()}
    # learned networks
    for name, net in nets.items():
        # warm-up (graph capture, lazy set-up) on a short run
        _timed_rollout(q0[: min(members, 8)].contiguous(), dt, [2], net=net, keep=False, stream=bs)
        flags, seg_ms = [], []
        states, ms, bad = _timed_rollout(q0, dt, segs, net=net, stream=bs, flags=flags, seg_ms=seg_ms)
        learned_ms = ms
        flagged = [int((f != 0).sum()) for f in flags]
        first_bad = {}
        for k, f in enumerate(flags):
            for b in np.nonzero(f)[0].tolist():
                first_bad.setdefault(b, k)
        if first_bad:
            idx = sorted(first_bad)
            qb = q0[idx].contiguous()
            pstates, pms, _ = _timed_rollout(qb, dt, segs, stream=bs)
            ms += pms
            for j, b in enumerate(idx):
                for k in range(first_bad[b], len(segs)):
                    states[k][b] = pstates[k][j]
            del pstates
        rate = members * n * n * horizons[-1] / (ms * 1e-3)
        res = {"cell_updates_per_s": rate, "seconds": ms * 1e-3,
               "learned_only_cell_updates_per_s": members * n * n * horizons[-1] / (learned_ms * 1e-3),
               "flagged_unstable_after_each_horizon": flagged,
               "members_on_plain_fallback": len(first_bad), "by_horizon": {}}
        for K, st, ref in zip(horizons, states, refs):
            acc = _ErrAcc(scale)
            acc.add(st, ref)
            e = acc.result()
            row = {"learned": e}
            for metric in ("scaled_rms", "e1_mean_rel_h"):
                errs = {N: (v["errors"][horizons.index(K)][metric]) for N, v in plain.items()}
                row[f"plain_{metric}"] = {str(N): v for N, v in errs.items()}
                row[f"n_eq_{metric}"] = _interp_resolution(errs, e[metric])
            res["by_horizon"][str(K)] = row
        del states
        # per horizon: N_eq by the scaled RMS, and the plain solver timed at
        # N_eq itself; where the learned error is below every plain error
        # measured, the largest N is a lower bound on N_eq (and the rate
        # comparison there a lower bound on the learned solver's advantage)
        res["accuracy_matched_by_horizon"] = {}
        for K in horizons:
            hrow = res["by_horizon"][str(K)]
            n_eq = hrow["n_eq_scaled_rms"]
            plain_err = {N: v["errors"][horizons.index(K)]["scaled_rms"] for N, v in plain.items()}
            bound = False
            if n_eq is None and hrow["learned"]["scaled_rms"] < min(plain_err.values()):
                n_eq, bound = float(max(plain_err)), True
            # the learned solver's rate up to K: its own steps so far, plus the
            # members that fell back by K run on the plain step at its 256^2 rate
            kk = horizons.index(K)
            fell = sum(1 for k in first_bad.values() if k <= kk)
            t_k = 1e-3 * sum(seg_ms[:kk + 1]) + fell * n * n * K / plain[n]["cell_updates_per_s"]
            rate_k = members * n * n * K / t_k
            mk = {"horizon": K, "metric": "scaled_rms", "n_eq": n_eq, "n_eq_is_lower_bound": bound,
                  "learned_rate": rate_k, "learned_error": hrow["learned"]["scaled_rms"],
                  "plain_error_same_n": plain_err[n], "members_on_fallback": fell}
            if n_eq is not None:
                r = n_eq / n
                N4 = max(8, int(round(n_eq / 4.0)) * 4)
                qN = _tiled_state(N4, seed, members, tiles)
                steps = max(2, int(round(K * N4 / n)))
                _, pms, _ = _timed_rollout(qN, dt * n / N4, [steps], keep=False, stream=bs)
                del qN
                prate = members * N4 * N4 * steps / (pms * 1e-3)
                mk.update({"r": r, "learned_rate_times_r3": rate_k * r ** 3, "plain_n_timed": N4,
                           "plain_rate_at_n_eq": prate, "learned_wins": rate_k * r ** 3 > prate})
            else:
                mk.update({"r": None, "learned_wins": False})
            res["accuracy_matched_by_horizon"][str(K)] = mk
        m = res["accuracy_matched_by_horizon"][str(headline)]
        res["accuracy_matched"] = m
        out[name] = res
        torch.cuda.empty_cache()
    return out


def save_weights(path: str, net, ds: Dataset, result: TrainResult, extra: dict | None = None,
                 norm=None) -> None:
    """Parameters, input normalisation (the network's own, `norm` = (mean,
    scale), else that of the dataset) and the training recipe in one .npz."""
    mean, scale = norm if norm is not None else input_scale(ds)
    meta = {"n_fine": ds.n_fine, "factor": ds.factor, "dt_coarse": ds.dt_coarse, "dt_fine": ds.dt_fine,
            "seed": ds.seed, "iters": result.iters,
            "final_loss": float(np.mean(result.losses[-50:])) if result.losses else None,
            "train_seconds": result.seconds}
    meta.update(extra or {})
    np.savez(path, params=fv.stencil_net_get_params(net), mean=mean, scale=scale,
             meta=np.array(repr(meta)), kind=np.array(net.kind))


def load_weights(path: str):
    """(net, metadata) from a file written by save_weights."""
    d = np.load(path, allow_pickle=False)
    kind = str(d["kind"]) if "kind" in d.files else "stencil"
    create = fv.face_net_create if kind == "face" else fv.stencil_net_create
    net = create(d["params"], d["mean"], d["scale"])
    import ast
    return net, ast.literal_eval(str(d["meta"]))


def load_norm(path: str):
    """(mean, scale) of the input normalisation stored with a network."""
    d = np.load(path, allow_pickle=False)
    return d["mean"], d["scale"]


def time_iterations(iters: int, kind: str = "stencil") -> float:
    """Milliseconds per training iteration of the bench's configuration (batch
    64 windows of 64^2, T = 8), after 3 warm-up iterations; the timed ones run
    inside the NVTX range "iter" (for a profiler's range filter)."""
    tr = generate(256, 4, members=64, seed=0, coarse_steps=32)
    if kind == "face":
        net = fv.face_net_create(init_params(0, kind="face", depth=float(data_stats(tr)[0][0])), *input_scale(tr))
    else:
        net = fv.stencil_net_create(init_params(0), *input_scale(tr))
    train(tr, iters=3, batch=64, T=8, net=net)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("iter")
    res = train(tr, iters=iters, batch=64, T=8, net=net)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    return 1e3 * res.seconds / iters


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="train the learned-stencil network on GPU-generated data")
    ap.add_argument("--members", type=int, default=256)
    ap.add_argument("--coarse-steps", type=int, default=256)
    ap.add_argument("--iters", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--T", type=int, default=8)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--kind", choices=["stencil", "face"], default="stencil")
    ap.add_argument("--pushforward", type=int, default=0,
                    help="untaped learned steps (at most) before each window's taped steps")
    ap.add_argument("--init", default=None,
                    help="continue from a saved network (its parameters, normalisation and dt)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--time-iterations", type=int, default=0,
                    help="only time this many training iterations (bench configuration) and exit")
    a = ap.parse_args(argv)
    if a.time_iterations:
        print(f"ms per iteration {time_iterations(a.time_iterations, a.kind):.3f}")
        return
    if not a.out:
        ap.error("--out is required")
    net, norm, dt_fine, extra = None, None, None, {}
    if a.init:
        net, meta0 = load_weights(a.init)
        norm = load_norm(a.init)
        dt_fine = meta0["dt_fine"]
        extra = {"init": {k: meta0[k] for k in ("iters", "final_loss") if k in meta0}}
    ds = generate(256, 4, members=a.members, seed=0, coarse_steps=a.coarse_steps, dt_fine=dt_fine)
    res = train(ds, iters=a.iters, batch=a.batch, T=a.T, lr=a.lr, seed=0, log_every=100, kind=a.kind,
                net=net, pushforward=a.pushforward)
    te = generate(256, 4, members=32, seed=2, coarse_steps=128, dt_fine=ds.dt_fine)
    _, std = data_stats(ds)
    ev = {k: evaluate(res.net, te, k, std) for k in (16, 64, 128)}
    print({k: (v["learned"], v["plain"]) for k, v in ev.items()})
    extra.update({"T": a.T, "coarse_steps": a.coarse_steps, "lr": a.lr, "pushforward": a.pushforward,
                  "rejected": res.rejected,
                  "test_errors": {k: (v["learned"], v["plain"]) for k, v in ev.items()}})
    save_weights(a.out, res.net, ds, res, extra, norm=norm)


if __name__ == "__main__":
    main()
