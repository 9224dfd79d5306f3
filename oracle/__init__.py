"""FP64 CPU oracle — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct restatement of what the thesis's finite-volume
method computes, written from the equations in its Section 2 (Eqs. 2.3-2.5,
2.9, 2.10, 2.15, 2.18, 2.19, 2.23, 2.24, 2.28, 5.1) and Section 2.5.3 (the
learned reconstruction-slope coefficients).  Plain PyTorch CPU tensor ops in
float64; periodic neighbours are ``torch.roll``; no blocking, fusion or
reordering beyond what the equations state.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and imports nothing from it; inputs come from the separate seeded
generator module ``paper_2602_08670_gb300.workloads``.

Modules
-------
fv           plain MUSCL-minmod + HLL + SSP-RK2 step for 2D SWE and 2D Euler,
             CFL time step, FP64 diagnostics, coarse graining.
riemann      exact Riemann solutions (shallow-water dam break, Sod) used as pins.
stencil_net  the learned-stencil variant: CNN, coefficient normalisation,
             learned reconstruction with minmod fallback, rollout loss (2.28);
             its gradients come from reverse-mode differentiation of this FP64
             forward and are pinned by central finite differences.
schemes      the other numerical fluxes (Lax-Friedrichs, Rusanov, Roe, HLLE,
             HLLC) and SSP-RK3.
bathymetry   the bed-slope source and reflecting walls (shallow water and
             Euler).
face_net     the face-state network (third data-driven approach): GeLU CNN,
             Softplus depths, side states paired at faces, rollout gradients.
sphere       shallow water on the sphere: the two-hemisphere grid and its
             metrics, rotated fluxes, curvature correction, Coriolis and
             tangent projection.
"""
