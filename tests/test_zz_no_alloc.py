"""fv_diagnostics_noalloc: the FP64 diagnostics for callers that cannot
allocate device memory while running (fixed memory budget, allocation-free
loops or callbacks, frameworks owning all device memory).  Its result must
equal that of the allocating fv_diagnostics on the same state, call after
call, although every call shares the library's fixed scratch array.  This
file is collected last so that a failure here comes after every other test."""
import ctypes

import numpy as np
import pytest
import torch

from helpers import f32
from paper_2602_08670_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_08670_gb300 import fv as binding
    return binding


def _noalloc(fv, q, eq, phys, loc):
    B, C, ny, nx = q.shape
    L = fv.lib()
    if loc == fv.FV_HOST:
        out = np.zeros((B, C + 1), dtype=np.float64)
        ptr = out.ctypes.data_as(ctypes.c_void_p)
    else:
        out = torch.zeros((B, C + 1), dtype=torch.float64, device="cuda")
        ptr = ctypes.c_void_p(out.data_ptr())
    torch.cuda.synchronize()
    rc = L.fv_diagnostics_noalloc(ctypes.c_void_p(q.data_ptr()), eq, B, ny, nx, 1.0, 1.0, phys, ptr,
                                  loc, None)
    assert rc == 0, L.fv_last_error()
    if loc == fv.FV_DEVICE:
        torch.cuda.synchronize()
        out = out.cpu().numpy()
    return out


def test_noalloc_diagnostics_match_allocating_entry_point(fv):
    # call 1: a batch of 3 shallow-water members after some steps
    q0 = f32(W.random_smooth_swe(64, seed=12, members=3, vel=0.2)[:, :, :48, :])
    s = fv.swe_init(q0.cuda())
    fv.fv_rollout(s, 10)
    ref = fv.fv_diagnostics(s)
    got = _noalloc(fv, fv.fv_get_state(s), 0, 9.81, fv.FV_HOST)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-14), (got, ref)
    # call 2, right after: an Euler batch (different shape), device output
    e0 = f32(np.concatenate([W.euler_kelvin_helmholtz(96, 64, seed=k) for k in range(2)]))
    es = fv.euler_init(e0.cuda())
    fv.fv_rollout(es, 5)
    eref = fv.fv_diagnostics(es)
    egot = _noalloc(fv, fv.fv_get_state(es), 1, 1.4, fv.FV_DEVICE)
    assert np.allclose(egot, eref, rtol=1e-12, atol=1e-14), (egot, eref)
    # and the first state again: nothing left over from the previous call matters
    again = _noalloc(fv, fv.fv_get_state(s), 0, 9.81, fv.FV_HOST)
    assert np.allclose(again, ref, rtol=1e-12, atol=1e-14)


def test_noalloc_rejects_batches_beyond_the_fixed_scratch(fv):
    L = fv.lib()
    q = torch.ones((81, 3, 8, 8), dtype=torch.float32, device="cuda")
    out = np.zeros((81, 4))
    rc = L.fv_diagnostics_noalloc(ctypes.c_void_p(q.data_ptr()), 0, 81, 8, 8, 1.0, 1.0, 9.81,
                                  out.ctypes.data_as(ctypes.c_void_p), fv.FV_HOST, None)
    assert rc == fv.FV_EINVAL
    assert b"scratch" in L.fv_last_error()


def _raw_call(fv, q, eq, B, phys):
    L = fv.lib()
    out = np.zeros((B, (3 if eq == 0 else 4) + 1))
    torch.cuda.synchronize()
    rc = L.fv_diagnostics_noalloc(ctypes.c_void_p(q.data_ptr()), eq, B, q.shape[2], q.shape[3], 1.0, 1.0,
                                  phys, out.ctypes.data_as(ctypes.c_void_p), fv.FV_HOST, None)
    return rc, out


def test_noalloc_capacity_limits_are_exact(fv):
    # 80 shallow-water members (80 x 4 slots) and 64 Euler members (64 x 5)
    # fill the 320 slots exactly and must match the allocating entry point;
    # one member more of either is rejected
    qs = f32(W.random_smooth_swe(16, seed=3, members=80, vel=0.2)).cuda()
    s = fv.swe_init(qs)
    fv.fv_rollout(s, 3)
    ref = fv.fv_diagnostics(s)
    rc, got = _raw_call(fv, fv.fv_get_state(s), 0, 80, 9.81)
    assert rc == fv.FV_OK, fv.lib().fv_last_error()
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-14)
    qe = f32(np.concatenate([W.euler_kelvin_helmholtz(16, 8, seed=k) for k in range(64)])).cuda()
    es = fv.euler_init(qe)
    fv.fv_rollout(es, 2)
    eref = fv.fv_diagnostics(es)
    rc, egot = _raw_call(fv, fv.fv_get_state(es), 1, 64, 1.4)
    assert rc == fv.FV_OK, fv.lib().fv_last_error()
    assert np.allclose(egot, eref, rtol=1e-12, atol=1e-14)
    q65 = torch.ones((65, 4, 8, 16), dtype=torch.float32, device="cuda")
    rc, _ = _raw_call(fv, q65, 1, 65, 1.4)
    assert rc == fv.FV_EINVAL
    assert b"scratch" in fv.lib().fv_last_error()
