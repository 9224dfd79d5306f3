"""Block domain decomposition on one GPU (several subdomains of one grid in
one process, rings refreshed by fv_halo_exchange): the interiors of the
decomposed run equal the undecomposed run bitwise, on the bench's full-size
plain workloads (SWE 4096^2 bump, Euler 2048^2 Kelvin-Helmholtz; adaptive dt
reduced over the subdomains) and on learned 256^2 batches split into row
slabs (stencil network on the fused kernel, face-state network on the
two-pass path; fixed dt).  Also: the ring strips that fv_halo_pack /
fv_halo_unpack move between processes, and the argument checks."""
import ctypes
import os

import numpy as np
import pytest
import torch

from helpers import ROOT
from paper_2602_08670_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import decomp, fv, train
    return fv, decomp, train


def _whole(fv, q0, eq, steps, net=None, dt_mode="adaptive", dt_fixed=0.0):
    init = fv.swe_init if eq == "swe" else fv.euler_init
    s = init(q0.clone(), cfl=0.5, dt_mode=dt_mode, dt_fixed=dt_fixed)
    fv.fv_enqueue_steps(s, steps, net=net)
    fv.fv_sync(s)
    return fv.fv_get_state(s), fv.fv_get_time(s), fv.fv_diagnostics(s)


@pytest.mark.parametrize("eq,n,px,py", [("swe", 4096, 2, 2), ("swe", 4096, 4, 1), ("euler", 2048, 2, 2),
                                        ("euler", 2048, 1, 4), ("swe", 200, 5, 2)])
def test_plain_blocks_equal_the_whole_grid(mods, eq, n, px, py):
    fv, decomp, _ = mods
    if eq == "swe":
        q0 = torch.tensor(W.swe_gaussian_bump(n, n), dtype=torch.float32).cuda()
    else:
        q0 = torch.tensor(W.euler_kelvin_helmholtz(n, n, seed=0), dtype=torch.float32).cuda()
    steps = 6
    ref, (t_ref, dt_ref, k_ref), d_ref = _whole(fv, q0, eq, steps)
    dom = decomp.LocalDomain(q0, eq, px, py, halo=2)
    dom.step(steps)
    dom.sync()
    got = dom.state()
    assert torch.equal(got, ref), float((got - ref).abs().max())
    t, dt, k = dom.time()
    assert np.array_equal(t, t_ref) and np.array_equal(dt, dt_ref) and np.array_equal(k, k_ref)
    assert np.allclose(dom.diagnostics(), d_ref, rtol=1e-12, atol=1e-12 * np.abs(d_ref).max())


@pytest.mark.parametrize("kind,py", [("stencil", 2), ("stencil", 4), ("face", 2)])
def test_learned_row_slabs_equal_the_whole_grid(mods, kind, py):
    fv, decomp, TR = mods
    wfile = "swe64_from256.npz" if kind == "stencil" else "face64_from256.npz"
    net, meta = TR.load_weights(os.path.join(ROOT, "paper_2602_08670_gb300", "weights", wfile))
    n, members, steps = 256, 8, 8
    dt = meta["dt_coarse"] * 64 / n
    q0 = torch.tensor(W.swe_random_bumps_tiled(n, 3, members, 4), dtype=torch.float32).cuda()
    ref, (t_ref, _, _), _ = _whole(fv, q0, "swe", steps, net=net, dt_mode="fixed", dt_fixed=dt)
    dom = decomp.LocalDomain(q0, "swe", 1, py, halo=6, dt_mode="fixed", dt_fixed=dt, learned=kind == "stencil")
    dom.step(steps, net=net)
    dom.sync()
    got = dom.state()
    assert torch.equal(got, ref), float((got - ref).abs().max())
    assert np.array_equal(dom.time()[0], t_ref)


def test_halo_strips_move_the_layout_windows(mods):
    fv, decomp, _ = mods
    n, px, py, h = 64, 2, 2, 2
    L = decomp.Layout.make(n, n, px, py, h)
    g = torch.Generator().manual_seed(4)
    qe = (1.0 + 0.1 * torch.rand((2, 3, L.ny_ext, L.nx_ext), generator=g)).cuda()
    s = fv.swe_init(qe.clone())
    fv.fv_set_halo(s, L.hx, L.hy)
    for side in range(4):
        k = fv.fv_halo_strip_floats(s, side)
        buf = torch.empty(k, device="cuda")
        fv.fv_halo_pack(s, 0, side, buf)
        fv.fv_sync(s)
        assert torch.equal(buf, L.strip(qe, side, True).contiguous().reshape(-1))
    # unpacking writes exactly the ring window of that side
    for side in range(4):
        k = fv.fv_halo_strip_floats(s, side)
        src = torch.arange(k, dtype=torch.float32, device="cuda") + 10.0 * side
        fv.fv_halo_unpack(s, 0, side, src)
        fv.fv_sync(s)
        ref = qe.clone()
        L.strip(ref, side, False).copy_(src.reshape(L.strip(ref, side, False).shape))
        qe = ref
        assert torch.equal(fv.fv_get_state(s), qe)


def test_halo_arguments_are_checked(mods):
    fv, decomp, _ = mods
    q = torch.ones((1, 3, 16, 16), device="cuda")
    s = fv.swe_init(q)
    with pytest.raises(fv.FvError):
        fv.fv_set_halo(s, 5, 0)             # ring wider than a quarter of the grid
    with pytest.raises(fv.FvError):
        fv.fv_enqueue_stage(s, 3)
    fv.fv_set_scheme(s, "roe", 2)
    with pytest.raises(fv.FvError):
        fv.fv_enqueue_stage(s, 1)           # stages of the HLL/SSP-RK2 step only
    a = fv.swe_init(q)
    e = fv.euler_init(torch.tensor(W.euler_kelvin_helmholtz(16, 16), dtype=torch.float32).cuda())
    arr = (ctypes.c_void_p * 2)(a.handle.value, e.handle.value)
    with pytest.raises(fv.FvError):
        fv.fv_halo_exchange(arr, 2, 1, 0)   # different equations
    b = fv.swe_init(q)
    arr = (ctypes.c_void_p * 2)(a.handle.value, b.handle.value)
    with pytest.raises(fv.FvError):
        fv.fv_halo_exchange(arr, 2, 1, 0)   # split without a ring
