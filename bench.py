#!/usr/bin/env python3
"""Throughput benchmark of the finite-volume hot path on GB300.

One *step* = one SSP-RK2 step (both stages, MUSCL-minmod + HLL) of the two
plain-solver workloads run back to back:
  * 2D Euler, 2048 x 2048 periodic, gamma = 1.4, Kelvin-Helmholtz shear layer;
  * 2D shallow water, 4096 x 4096 periodic, Gaussian bump (g = 9.81);
both FP32 with the adaptive CFL 0.5 time step.  The default step count is the
workload's horizon of 2000 steps.  `value` is cell-updates per second summed
over both grids (and over all ranks); one cell-update is one cell advanced by
one full SSP-RK2 step.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (the
only reference implementation there is), on a bounded sample per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s plain vs learned at matched L2 error; p50/p99 request latency"
UNIT = "cell-updates/s"
N_SWE = 4096
N_EULER = 2048
SWE_BYTES_PER_CELL_UPDATE = 60     # stage 1: 12 + 12; stage 2: 12 + 12 + 12 (FP32, C = 3)
EULER_BYTES_PER_CELL_UPDATE = 80   # C = 4
CHUNK = 32                          # steps per enqueue between timing events
WORKLOAD = "plain FV step: Euler KH 2048^2 + SWE Gaussian bump 4096^2, FP32, SSP-RK2, CFL 0.5"
WEIGHTS = os.path.join(ROOT, "paper_2602_08670_gb300", "weights", "swe64_from256.npz")
FACE_WEIGHTS = os.path.join(ROOT, "paper_2602_08670_gb300", "weights", "face64_from256.npz")
# Seed of the accuracy-matched evaluation field.  The fine-tuning runs behind
# the committed stencil network were compared on seed 3; the bench evaluates
# on a field that took no part in that choice.
EVAL_SEED = 5


def captured_traffic(key):
    """DRAM bytes per launch pair from a committed ncu capture, or None when
    the kernel sources have changed since the counters were taken."""
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(prof):
        return None
    with open(prof) as f:
        entry = json.load(f).get(key)
    if not entry:
        return None
    h = hashlib.sha256()
    for src in entry["sources"]:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    return entry["bytes"] if h.hexdigest() == entry["source_sha256"] else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def dist_env():
    from paper_2602_08670_gb300 import ranks
    return ranks.env()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        # median over samples under load (clock above idle)
        top = max(sm) if sm else 0.0
        loaded = [v for v in sm if v >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle (the reference arm, and the cpu_baseline of our arm)
# ---------------------------------------------------------------------------

def oracle_sample(steps: int, n_swe: int, n_euler: int):
    """Time the FP64 oracle as it stands: `steps` SSP-RK2 steps of an SWE
    bump n_swe^2 and an Euler KH n_euler^2.  Returns (cell-updates/s, seconds,
    threads)."""
    import torch

    from oracle import fv as ofv
    from paper_2602_08670_gb300 import workloads as W
    qs = torch.tensor(W.swe_gaussian_bump(n_swe, n_swe))
    qe = torch.tensor(W.euler_kelvin_helmholtz(n_euler, n_euler, seed=0))
    t0 = time.perf_counter()
    ofv.run(qs, ofv.SWE, steps)
    ofv.run(qe, ofv.EULER, steps)
    dt = time.perf_counter() - t0
    cells = (n_swe * n_swe + n_euler * n_euler) * steps
    return cells / dt, dt, torch.get_num_threads()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n_swe, n_euler = 128, 128
    oracle_sample(max(1, args.warmup), 32, 32)     # warm-up
    rate, secs, threads = oracle_sample(args.steps, n_swe, n_euler)
    sample = f"{args.steps} steps of SWE bump {n_swe}^2 + Euler KH {n_euler}^2 (FP64 oracle)"
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD + " (oracle on a bounded sample)"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv
    from paper_2602_08670_gb300 import ranks
    from paper_2602_08670_gb300 import workloads as W

    bs = torch.cuda.Stream()
    q_swe = torch.tensor(W.swe_gaussian_bump(N_SWE, N_SWE), dtype=torch.float32)
    q_eul = torch.tensor(W.euler_kelvin_helmholtz(N_EULER, N_EULER, seed=0), dtype=torch.float32)
    with torch.cuda.stream(bs):
        swe = fv.swe_init(q_swe.cuda(), cfl=0.5)
        eul = fv.euler_init(q_eul.cuda(), cfl=0.5)
    assert swe.stream == bs.cuda_stream and eul.stream == bs.cuda_stream

    def barrier():
        ranks.barrier()
        torch.cuda.synchronize()

    # warm-up (also captures the graphs)
    for _ in range(max(args.warmup, 3)):
        fv.fv_enqueue_steps(swe, 1)
        fv.fv_enqueue_steps(eul, 1)
    fv.fv_enqueue_steps(swe, CHUNK)
    fv.fv_enqueue_steps(eul, CHUNK)
    fv.fv_sync(swe)
    fv.fv_sync(eul)

    K = args.steps
    chunks = [CHUNK] * (K // CHUNK) + ([K % CHUNK] if K % CHUNK else [])
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in chunks]
    clocks = Clocks(local)
    clocks.start()
    barrier()
    for c, k in enumerate(chunks):
        ev[c][0].record(bs)
        fv.fv_enqueue_steps(swe, k)
        ev[c][1].record(bs)
        fv.fv_enqueue_steps(eul, k)
        ev[c][2].record(bs)
    barrier()
    clk = clocks.stop()
    total_ms = ev[0][0].elapsed_time(ev[-1][2])
    swe_ms = sum(e[0].elapsed_time(e[1]) for e in ev)
    eul_ms = sum(e[1].elapsed_time(e[2]) for e in ev)
    fv.fv_sync(swe)
    fv.fv_sync(eul)
    cells_per_step = N_SWE * N_SWE + N_EULER * N_EULER
    value, secs = ranks.job_rate(cells_per_step * K, total_ms * 1e-3, device="cuda")
    total_ms = secs * 1e3

    # roofline of the dominant kernel pair (SWE stage 1 + stage 2)
    peak, peak_kind = measured_peaks()
    swe_step_s = swe_ms * 1e-3 / K
    achieved = SWE_BYTES_PER_CELL_UPDATE * N_SWE * N_SWE / swe_step_s / 1e9
    eul_achieved = EULER_BYTES_PER_CELL_UPDATE * N_EULER * N_EULER / (eul_ms * 1e-3 / K) / 1e9
    traffic = captured_traffic("swe_stage_pair_4096")

    # end to end through the public API with host buffers: upload the initial
    # states from pinned memory, advance them by K steps, read the results back
    state_bytes = (q_swe.numel() + q_eul.numel()) * 4
    e2e = None
    if not args.no_e2e:
        h_swe = q_swe.pin_memory()
        h_eul = q_eul.pin_memory()
        o_swe = torch.empty_like(h_swe).pin_memory()
        o_eul = torch.empty_like(h_eul).pin_memory()
        e2e_runs = []
        for rep in range(2):
            barrier()
            t0 = time.perf_counter()
            fv.fv_set_state(swe, h_swe)
            fv.fv_set_state(eul, h_eul)
            fv.fv_enqueue_steps(swe, K)
            fv.fv_enqueue_steps(eul, K)
            fv.fv_get_state(swe, out=o_swe)
            fv.fv_get_state(eul, out=o_eul)
            barrier()
            e2e_runs.append(time.perf_counter() - t0)
        e2e_s = min(e2e_runs[1:]) if len(e2e_runs) > 1 else e2e_runs[0]
        e2e_rate, e2e_s = ranks.job_rate(cells_per_step * K, e2e_s, device="cuda")
        assert bool(torch.isfinite(o_swe).all()) and bool(torch.isfinite(o_eul).all())
        e2e = {"value": e2e_rate, "unit": UNIT,
               "h2d_bytes_per_step": state_bytes / K, "d2h_bytes_per_step": state_bytes / K,
               "call": "fv_set_state(host) + fv_enqueue_steps(K) + fv_get_state(host) per state"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "swe": f"{N_SWE}x{N_SWE} Gaussian bump h=1+0.1exp(-r^2/0.005)",
                   "euler": f"{N_EULER}x{N_EULER} Kelvin-Helmholtz, seed 0",
                   "per_rank": "each rank runs its own copy (independent problems)",
                   "l2": "inputs larger than L2 (SWE state buffer 201 MB > 129 MB L2)",
                   "swe_cell_updates_per_s": N_SWE * N_SWE * K / (swe_ms * 1e-3),
                   "euler_cell_updates_per_s": N_EULER * N_EULER * K / (eul_ms * 1e-3),
                   "euler_stage_pair_gbs": eul_achieved},
        "roofline": {"bound": "hbm", "kernel": "stage_march_kernel<SWE> (stage 1 + stage 2)",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_unit": "DRAM bytes per stage pair (ncu capture)",
                     "algorithmic_bytes": f"{SWE_BYTES_PER_CELL_UPDATE} B/cell-update x {N_SWE}^2 cells per step"},
        "e2e": e2e,
        "gpu_launches": 4 * K,
        "clocks": clk,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the bench's own grids (SWE 4096^2 + Euler 2048^2), four steps: about
        # ten seconds of FP64 work on the host cores
        rate, secs, threads = oracle_sample(4, N_SWE, N_EULER)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"4 SSP-RK2 steps of SWE bump {N_SWE}^2 + Euler KH {N_EULER}^2, "
                                          f"FP64 oracle, {secs:.1f} s"}
    if not args.no_schemes:
        line["schemes"] = schemes_block(args)
        line["sphere"] = sphere_block(args)
    if not args.no_learned:
        line["learned"] = learned_block(args)
    if not args.no_serving:
        lrate = line.get("learned", {}).get("accuracy_matched", {}).get("stencil", {}).get(
            "learned_only_cell_updates_per_s")
        line["serving"] = serving_block(args, N_SWE * N_SWE * K / (swe_ms * 1e-3), lrate)
    # compact summary of the learned and serving results as the line's last key
    line["summary"] = summary(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def learned_block(args):
    """The learned-stencil path.  `accuracy_matched`: each trained network's
    batched rollout on 256 members x 256^2 (fused tcgen05 kernel for the
    stencil network, CNN + face-state stage kernels for the face-state
    network), timed, with its state at every horizon compared against the
    plain solver at 1024^2 coarse-grained 4x; the plain solver at 256^2 ..
    768^2 gives the resolution N_eq of equal error and is timed there (the
    plain rate at matched accuracy).  Also: the CNN's tensor-pipe roofline
    from that rollout, the same rollout through the two-pass path, and one
    training iteration of each network (batch 64, 64^2, T = 8)."""
    import torch

    from paper_2602_08670_gb300 import fv
    from paper_2602_08670_gb300 import train as TR
    from paper_2602_08670_gb300 import workloads as W

    out = {}
    net, meta = TR.load_weights(WEIGHTS)
    fnet, _ = TR.load_weights(FACE_WEIGHTS)
    tr = TR.generate(256, 4, members=64, seed=0, coarse_steps=32)
    _, std = TR.data_stats(tr)
    horizons = tuple(int(k) for k in args.learned_horizons.split(","))
    m = TR.matched_accuracy({"stencil": net, "face_state": fnet}, meta["dt_coarse"], std, n=256, tiles=4,
                            members=args.learned_members, seed=EVAL_SEED, horizons=horizons)
    out["accuracy_matched"] = m
    bf16_peak = _bf16_sustained_peak()
    members, n = args.learned_members, 256
    rate = m["stencil"]["cell_updates_per_s"]
    tflops = 118656 * rate / 1e12
    out["rollout"] = {"workload": f"{members} members x {n}^2 SWE, stencil network, fixed dt, "
                                  f"{horizons[-1]} steps (the accuracy_matched run)",
                      "kernel": "learned_fused_kernel (CNN on tcgen05 + learned faces + HLL + RK, "
                                "one launch per stage)",
                      "cell_updates_per_s": rate, "cnn_tflops": tflops,
                      "roofline": {"bound": "tensor", "achieved": tflops, "peak": bf16_peak,
                                   "unit": "TFLOP/s", "frac": tflops / bf16_peak,
                                   "peak_kind": "measured bf16 sustained",
                                   "algorithmic": "118656 FLOP per cell-update (2 CNN passes of "
                                                  "59328 FLOP)"},
                      "hbm_gbs": 60 * rate / 1e9}
    frate = m["face_state"]["cell_updates_per_s"]
    out["face_state_rollout"] = {"kernel": "conv_kernel (GeLU / side-state epilogues) + stage_face_kernel",
                                 "cell_updates_per_s": frate, "cnn_tflops": 91008 * frate / 1e12,
                                 "roofline": {"bound": "tensor", "achieved": 91008 * frate / 1e12,
                                              "peak": bf16_peak, "unit": "TFLOP/s",
                                              "frac": 91008 * frate / 1e12 / bf16_peak,
                                              "peak_kind": "measured bf16 sustained"},
                                 "algorithmic": "91008 FLOP per cell-update (2 CNN passes of 45504 FLOP)"}
    # the stencil network's rollout through the two-pass path (CNN coefficients via HBM)
    q0 = torch.tensor(W.swe_random_bumps_tiled(n, 3, 32, 4), dtype=torch.float32).cuda()
    bs = torch.cuda.Stream()
    with torch.cuda.stream(bs):
        st = fv.swe_init(q0, dt_mode="fixed", dt_fixed=meta["dt_coarse"] * 64 / n)
    fv.fv_set_learned_variant(st, "two_pass")
    fv.fv_enqueue_steps(st, 2, net=net)
    fv.fv_sync(st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(bs)
    fv.fv_enqueue_steps(st, 10, net=net)
    e1.record(bs)
    fv.fv_sync(st)
    out["rollout"]["two_pass_cell_updates_per_s"] = 32 * n * n * 10 / (e0.elapsed_time(e1) * 1e-3)
    del st
    # one training iteration of each network (C3 shape)
    tnet = fv.stencil_net_create(TR.init_params(0), *TR.input_scale(tr))
    TR.train(tr, iters=3, batch=64, T=8, net=tnet)       # warm-up
    res = TR.train(tr, iters=10, batch=64, T=8, net=tnet)
    it_ms = 1e3 * res.seconds / res.iters
    # forward 2 passes x 59328 FLOP per cell and stage-1/2 ... per step; backward ~2x forward
    fwd = 64 * 64 * 64 * 16 * 59328
    burst = _bf16_burst_peak()
    tfl = 3 * fwd / (it_ms * 1e-3) / 1e12
    out["training"] = {"workload": "batch 64 windows, 64^2, T = 8 steps (16 stages), forward + "
                                   "Eq. 2.28 loss + backward + Adam",
                       "ms_per_iteration": it_ms,
                       "cnn_flop_per_iteration": 3 * fwd,
                       "roofline": {"bound": "tensor", "achieved": tfl, "peak": burst, "unit": "TFLOP/s",
                                    "frac": tfl / burst, "peak_kind": "measured bf16 burst",
                                    "algorithmic": "59328 FLOP per cell and CNN pass x 64 windows x 64^2 "
                                                   "cells x 16 stages, x3 with the backward"}}
    fnet_t = fv.face_net_create(TR.init_params(0, kind="face", depth=float(TR.data_stats(tr)[0][0])),
                                *TR.input_scale(tr))
    TR.train(tr, iters=3, batch=64, T=8, net=fnet_t)
    res = TR.train(tr, iters=10, batch=64, T=8, net=fnet_t)
    out["face_state_training"] = {"ms_per_iteration": 1e3 * res.seconds / res.iters}
    return out


def _bf16_burst_peak() -> float:
    """Measured burst BF16 tensor throughput (TFLOP/s), else the recipe's
    fallback."""
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        with open(pp) as f:
            return float(json.load(f).get("bf16_tflops", 1900.0))
    return 1900.0


def _bf16_sustained_peak() -> float:
    """Measured sustained BF16 tensor throughput (TFLOP/s), else the recipe's
    fallback."""
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        with open(pp) as f:
            return float(json.load(f).get("bf16_tflops_sustained", 1700.0))
    return 1700.0


def _sig(x, k=3):
    """x rounded to k significant digits (None and bools unchanged)."""
    if x is None or isinstance(x, bool) or not isinstance(x, (int, float)):
        return x
    return float(f"{x:.{k}g}")


def summary(line) -> dict:
    """The learned-vs-plain accuracy-matched numbers per horizon and the
    serving latencies, compact, for the end of the JSON line."""
    out = {"plain_cell_updates_per_s": _sig(line["value"])}
    lm = line.get("learned", {}).get("accuracy_matched")
    if lm:
        for name in ("stencil", "face_state"):
            out[name] = {K: [_sig(a["learned_error"], 2), _sig(a["plain_error_same_n"], 2),
                             (">" if a["n_eq_is_lower_bound"] else "") + str(_sig(a["n_eq"])),
                             _sig(a["learned_rate"], 2), _sig(a.get("learned_rate_times_r3"), 2),
                             _sig(a.get("plain_rate_at_n_eq"), 2), a["learned_wins"], a["members_on_fallback"]]
                         for K, a in lm[name]["accuracy_matched_by_horizon"].items()}
        out["legend"] = ("horizon: [learned err, plain err at 256^2, N_eq, learned cu/s, learned cu/s x "
                         "(N_eq/256)^3, plain cu/s at N_eq, learned wins, members on fallback]")
    sv = line.get("serving")
    if sv:
        out["serving"] = {"capacity_cell_updates_per_s": _sig(sv["capacity"]["throughput_cell_updates_per_s"]),
                          "kernel_bound": _sig(sv.get("kernel_bound_cell_updates_per_s")),
                          "p50_p99_s": {str(d["rate_fraction_of_capacity"]):
                                        [_sig(d["p50_latency_s"]), _sig(d["p99_latency_s"]), d["requests"]]
                                        for d in sv["load"]}}
    return out


def schemes_block(args):
    """The plain step with the other fluxes (Eqs. 2.11-2.17) and SSP-RK3
    (Eq. 2.20) on the SWE 4096^2 bump: rate and HBM roofline of the row-march
    stage kernel with the flux chosen per launch, and of the shared-memory
    tile kernel for one scheme (algorithmic bytes 60 per cell-update for
    SSP-RK2, 96 for SSP-RK3: stage 1 reads q^n and writes q1, the others read
    their input and q^n and write).  The bathymetry entry is Section 4.2's
    configuration on the same grid: a Perlin-noise bed (Eq. 2.3's source),
    reflecting walls and Roe with SSP-RK2 in the row-march kernel, 68 bytes
    per cell-update (each stage also reads the bed)."""
    import torch

    from paper_2602_08670_gb300 import fv
    from paper_2602_08670_gb300 import workloads as W

    peak, _ = measured_peaks()
    q0 = torch.tensor(W.swe_gaussian_bump(N_SWE, N_SWE), dtype=torch.float32).cuda()
    bs = torch.cuda.Stream()
    out = {"workload": f"SWE Gaussian bump {N_SWE}^2, CFL 0.5 adaptive dt, 20 steps per scheme",
           "kernel": "stage_march_kernel (generic instances, flux chosen per launch); "
                     "_tile: stage_scheme_kernel (shared-memory tile)"}
    K = 20
    runs = [(f, r, "march") for f, r in (("rusanov", 2), ("lf", 2), ("roe", 2), ("hlle", 2), ("hllc", 2),
                                         ("hll", 3), ("hllc", 3))] + [("hllc", 2, "tile"), ("roe", 2, "bathymetry")]
    z = torch.tensor(W.perlin_bed(N_SWE, N_SWE, seed=11), dtype=torch.float32).cuda()
    qb = torch.tensor(W.swe_bump_over_bed(z.double().cpu().numpy()), dtype=torch.float32).cuda()
    for flux, rk, variant in runs:
        bed = variant == "bathymetry"
        with torch.cuda.stream(bs):
            st = fv.swe_init((qb if bed else q0).clone(), cfl=0.5)
        fv.fv_set_scheme(st, flux, rk)
        if bed:
            fv.fv_set_boundary(st, "wall")
            fv.fv_set_bathymetry(st, z)
        else:
            fv.fv_set_stage_variant(st, variant)
        fv.fv_enqueue_steps(st, 3)
        fv.fv_sync(st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(bs)
        fv.fv_enqueue_steps(st, K)
        e1.record(bs)
        fv.fv_sync(st)
        ms = e0.elapsed_time(e1)
        rate = N_SWE * N_SWE * K / (ms * 1e-3)
        gbs = (68 if bed else 60 if rk == 2 else 96) * rate / 1e9
        key = "bathymetry_walls_roe_rk2" if bed else f"{flux}_rk{rk}" + ("_tile" if variant == "tile" else "")
        out[key] = {"cell_updates_per_s": rate, "ms_per_step": ms / K,
                    "hbm_gbs": gbs, "frac_of_measured_hbm": gbs / peak}
        del st
    # Section 4.2's planar Euler test: a four-quadrant Riemann problem between
    # walls (seeded states), HLLE with SSP-RK2, 80 bytes per cell-update
    qe = torch.tensor(W.euler_four_quadrant(N_EULER, N_EULER, seed=4), dtype=torch.float32).cuda()
    with torch.cuda.stream(bs):
        st = fv.euler_init(qe, cfl=0.5)
    fv.fv_set_scheme(st, "hlle", 2)
    fv.fv_set_boundary(st, "wall")
    fv.fv_enqueue_steps(st, 3)
    fv.fv_sync(st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bs)
    fv.fv_enqueue_steps(st, K)
    e1.record(bs)
    fv.fv_sync(st)
    ms = e0.elapsed_time(e1)
    rate = N_EULER * N_EULER * K / (ms * 1e-3)
    out["euler_four_quadrant_walls_hlle_rk2"] = {
        "workload": f"Euler four-quadrant Riemann problem {N_EULER}^2, walls, CFL 0.5",
        "cell_updates_per_s": rate, "ms_per_step": ms / K, "hbm_gbs": 80 * rate / 1e9,
        "frac_of_measured_hbm": 80 * rate / 1e9 / peak}
    del st
    return out


def sphere_block(args):
    """Shallow water on the sphere (Sections 2.4, 4.3) on the thesis's
    finest grid, 1000 x 500 cells: one member (the thesis's run) and a
    batch of 32 members sharing the grid metrics, with HLL, and one member
    with Roe (the thesis's flux for its sphere runs).  Algorithmic HBM bytes per
    cell-update: 80 for the state (stage 1 reads q^n, writes q1; stage 2
    reads q1 and q^n, writes q^{n+1}; 16 B per cell each) plus the metrics,
    232 B per cell and step (x and y faces 40 B each, cells 36 B, read by
    both stages), shared by the batch."""
    import torch

    from paper_2602_08670_gb300 import fv
    from paper_2602_08670_gb300 import workloads as W

    peak, _ = measured_peaks()
    g_nd, omega = 11489.57, 6.300388          # Earth radii and days
    nx, ny = 1000, 500
    out = {"workload": f"sphere {nx} x {ny}, seeded bumps + rigid rotation, HLL SSP-RK2, CFL 0.5, "
                       "g and Omega in Earth radii / days",
           "kernel": "sphere_stage_kernel (tile, 4 variables, rotated HLL + correction + Coriolis + projection)"}
    bs = torch.cuda.Stream()
    for members, K, flux in ((1, 50, "hll"), (32, 10, "hll"), (1, 50, "roe")):
        with torch.cuda.stream(bs):
            st = fv.sphere_init(torch.ones(1, 4, ny, nx, device="cuda"), g=g_nd, omega=omega)
        c, _ = fv.sphere_get_cells(st)
        del st
        q0 = torch.tensor(W.sphere_bumps(c, 5, members, spin=1.0), dtype=torch.float32).cuda()
        with torch.cuda.stream(bs):
            st = fv.sphere_init(q0, g=g_nd, omega=omega)
        fv.fv_set_scheme(st, flux, 2)
        fv.fv_enqueue_steps(st, 3)
        fv.fv_sync(st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(bs)
        fv.fv_enqueue_steps(st, K)
        e1.record(bs)
        fv.fv_sync(st)
        ms = e0.elapsed_time(e1)
        rate = members * nx * ny * K / (ms * 1e-3)
        bytes_per = 80 + 232 / members
        key = f"members_{members}" + ("" if flux == "hll" else f"_{flux}")
        out[key] = {"cell_updates_per_s": rate, "ms_per_step": ms / K,
                                     "algorithmic_bytes_per_cell_update": bytes_per,
                                     "hbm_gbs": bytes_per * rate / 1e9,
                                     "frac_of_measured_hbm": bytes_per * rate / 1e9 / peak}
        del st
    return out


def serving_block(args, plain_rate=None, learned_rate=None):
    """Continuous-batching server under Poisson load: requests of SWE (50 %
    learned, 25 % plain) and Euler (25 %), grids uniform over {64, 128, 256,
    512}^2, horizons uniform in [100, 1000] (a reduced version of the full
    serving workload, which has grids to 2048^2 and horizons to 5000 steps;
    `python -m paper_2602_08670_gb300.serve` runs that).  Capacity = requests
    per second with all requests queued at t = 0; the Poisson runs use 0.5,
    0.9 and 1.2 x capacity.  The kernel bound is the throughput the same mix
    reaches at the plain and learned kernels' full-GPU rates."""
    from paper_2602_08670_gb300 import fv, serve
    from paper_2602_08670_gb300 import train as TR
    from paper_2602_08670_gb300 import workloads as W

    net, _ = TR.load_weights(WEIGHTS)
    base = W.serving_requests(args.serve_requests, 1.0, seed=42, sizes=(64, 128, 256, 512),
                              horizon=(100, 1000))
    server = fv.fv_server_create(64 << 30, 256, net)
    out = {"workload": f"{args.serve_requests} requests per rate: 50 % learned SWE, 25 % plain SWE, "
                       "25 % plain Euler; grids {64,128,256,512}^2; horizons U[100,1000]; seed 42; "
                       "budget 64 GB, 256 slots"}
    out.update(serve.sweep(server, base, (0.5, 0.9, 1.2)))
    if plain_rate and learned_rate:
        out["kernel_bound_cell_updates_per_s"] = serve.kernel_bound(base, plain_rate, learned_rate)
    out["learned_fallbacks_to_plain"] = fv.fv_server_stats(server)[3]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end run")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-path measurements")
    ap.add_argument("--learned-horizons", default="64,256,1000,2000",
                    help="coarse steps at which the learned rollout is compared with the reference")
    ap.add_argument("--learned-members", type=int, default=256)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurements")
    ap.add_argument("--no-schemes", action="store_true",
                    help="skip the other fluxes / SSP-RK3 measurements")
    ap.add_argument("--serve-requests", type=int, default=128)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
