"""Time a batched rollout of the learned (or plain) shallow-water step.

    python -m paper_2602_08670_gb300.rollout --members 64 --n 256 --steps 3 --variant fused
    python -m paper_2602_08670_gb300.rollout --members 16 --n 1024 --variant plain --flux hllc --rk 3
    python -m paper_2602_08670_gb300.rollout --members 64 --n 256 --steps 3 --variant face

Members are the random-bump initial states of `workloads.swe_random_bumps`
(seed 3), the network the committed trained weights (the stencil network, or
with ``--variant face`` the face-state network), dt the fine time step they
were trained with.  The plain variant takes any flux and integrator of
`fv.fv_set_scheme` and the adaptive dt of CFL 0.5 (the fine time step is
stable only on the 256^2 grid it was trained on).  Prints the wall-clock time per step and the rate in
cell-updates per second.
"""
from __future__ import annotations

import argparse
import os
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--variant", choices=["auto", "fused", "two_pass", "plain", "face"], default="fused")
    ap.add_argument("--flux", choices=["hll", "rusanov", "lf", "roe", "hlle", "hllc"], default="hll",
                    help="numerical flux of the plain variant")
    ap.add_argument("--rk", type=int, choices=[2, 3], default=2, help="integrator of the plain variant")
    args = ap.parse_args(argv)

    import torch

    from . import build, fv, train, workloads

    build.build()
    wname = "face64_from256.npz" if args.variant == "face" else "swe64_from256.npz"
    net, meta = train.load_weights(os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", wname))
    q0 = torch.tensor(workloads.swe_random_bumps(args.n, 3, args.members), dtype=torch.float32).cuda()
    use = None if args.variant == "plain" else net
    if use is not None:
        st = fv.swe_init(q0, dt_mode="fixed", dt_fixed=meta["dt_fine"])
        if args.variant != "face":
            fv.fv_set_learned_variant(st, args.variant)
    else:
        st = fv.swe_init(q0, cfl=0.5)
        fv.fv_set_scheme(st, args.flux, args.rk)
    fv.fv_enqueue_steps(st, 2, net=use)
    fv.fv_sync(st)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fv.fv_enqueue_steps(st, args.steps, net=use)
    fv.fv_sync(st)
    dt = time.perf_counter() - t0
    cells = args.members * args.n * args.n * args.steps
    name = args.variant if use is not None else f"plain {args.flux} rk{args.rk}"
    print(f"{name} {args.members} x {args.n}^2, {args.steps} steps: {1e3 * dt / args.steps:.3f} ms/step, "
          f"{cells / dt:.4g} cell-updates/s")


if __name__ == "__main__":
    main()
