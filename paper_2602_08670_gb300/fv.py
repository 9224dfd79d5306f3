"""Python binding of libfv (include/fv.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts torch
tensors to pointers, picks the location tag, and turns negative status codes
into ``FvError``.  Functions carry the C names.  Loading fails loudly when
``libfv.so`` has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from .build import LIB

c_int, c_long, c_double, c_void_p = ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_void_p

FV_OK, FV_PENDING = 0, 1
FV_EINVAL, FV_ENOMEM, FV_EUNSTABLE, FV_ETIMEOUT, FV_EBUSY, FV_ECUDA, FV_ENOTFOUND = range(-1, -8, -1)
FV_HOST, FV_DEVICE = 0, 1
DT_MODES = {"adaptive": 0, "fixed": 1, "replay": 2}
STATUS_NAMES = {0: "FV_OK", 1: "FV_PENDING", -1: "FV_EINVAL", -2: "FV_ENOMEM", -3: "FV_EUNSTABLE",
                -4: "FV_ETIMEOUT", -5: "FV_EBUSY", -6: "FV_ECUDA", -7: "FV_ENOTFOUND"}
CUDA_STREAM_LEGACY = 1


class FvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class fv_grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("batch", c_int), ("lx", c_double), ("ly", c_double)]


class fv_swe_params(ctypes.Structure):
    _fields_ = [("g", c_double), ("cfl", c_double), ("dt_mode", c_int), ("dt_fixed", c_double)]


class fv_euler_params(ctypes.Structure):
    _fields_ = [("gamma", c_double), ("cfl", c_double), ("dt_mode", c_int), ("dt_fixed", c_double)]


class fv_sphere_params(ctypes.Structure):
    _fields_ = [("g", c_double), ("omega", c_double), ("cfl", c_double), ("dt_mode", c_int),
                ("dt_fixed", c_double)]


_lib = None

# name -> argtypes (all functions return int unless listed in _RESTYPES)
_SIGS = {
    "fv_last_error": [],
    "swe_init": [ctypes.POINTER(fv_grid), ctypes.POINTER(fv_swe_params), c_void_p, c_int, c_void_p,
                 ctypes.POINTER(c_void_p)],
    "euler_init": [ctypes.POINTER(fv_grid), ctypes.POINTER(fv_euler_params), c_void_p, c_int,
                   c_void_p, ctypes.POINTER(c_void_p)],
    "fv_destroy_state": [c_void_p],
    "sphere_init": [c_int, c_int, c_int, ctypes.POINTER(fv_sphere_params), c_void_p, c_int, c_void_p,
                    ctypes.POINTER(c_void_p)],
    "sphere_get_cells": [c_void_p, c_void_p, c_void_p, c_int],
    "fv_set_replay_dt": [c_void_p, c_void_p, c_long],
    "fv_step": [c_void_p, c_void_p],
    "fv_rollout": [c_void_p, c_void_p, c_long, c_double, c_void_p, c_int, c_int, c_void_p],
    "fv_enqueue_steps": [c_void_p, c_void_p, c_long],
    "fv_sync": [c_void_p],
    "fv_get_state": [c_void_p, c_void_p, c_int],
    "fv_set_state": [c_void_p, c_void_p, c_int],
    "fv_state_device_ptr": [c_void_p, ctypes.POINTER(c_void_p)],
    "fv_state_stream": [c_void_p, ctypes.POINTER(c_void_p)],
    "fv_set_stage_variant": [c_void_p, c_int],
    "fv_set_learned_variant": [c_void_p, c_int],
    "fv_set_scheme": [c_void_p, c_int, c_int],
    "fv_set_boundary": [c_void_p, c_int],
    "fv_set_bathymetry": [c_void_p, c_void_p, c_int],
    "fv_set_learned_hmin": [c_void_p, c_double],
    "stencil_net_create": [c_void_p, c_void_p, ctypes.POINTER(c_void_p)],
    "stencil_net_destroy": [c_void_p],
    "stencil_net_set_params": [c_void_p, c_void_p, c_int],
    "stencil_net_get_params": [c_void_p, c_void_p, c_int],
    "stencil_net_forward": [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_int, c_void_p],
    "face_net_create": [c_void_p, c_void_p, ctypes.POINTER(c_void_p)],
    "stencil_net_backward": [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p],
    "face_net_backward": [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p],
    "face_net_forward": [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_int, c_void_p],
    "fv_net_kind": [c_void_p],
    "fv_net_num_params": [c_void_p],
    "fv_tape_create": [c_void_p, c_int, c_int, c_int, c_int, c_double, c_double, c_double,
                       ctypes.POINTER(c_void_p)],
    "fv_tape_destroy": [c_void_p],
    "fv_tape_forward": [c_void_p, c_void_p, c_void_p],
    "fv_tape_loss": [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double)],
    "fv_tape_backward": [c_void_p, c_void_p, c_void_p, c_void_p],
    "stencil_net_adam_step": [c_void_p, c_void_p, c_int, c_double, c_double, c_double, c_double],
    "fv_coarsen": [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p],
    "fv_server_create": [ctypes.c_size_t, c_int, c_void_p, ctypes.POINTER(c_void_p)],
    "fv_server_destroy": [c_void_p],
    "fv_submit": [c_void_p, c_void_p, ctypes.POINTER(ctypes.c_ulonglong)],
    "fv_poll": [c_void_p, ctypes.c_ulonglong, c_void_p, ctypes.POINTER(c_double)],
    "fv_server_stats": [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                        ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_longlong)],
    "fv_diagnostics_noalloc": [c_void_p, c_int, c_int, c_int, c_int, c_double, c_double, c_double,
                               c_void_p, c_int, c_void_p],
    "fv_get_time": [c_void_p, c_void_p, c_void_p, c_void_p],
    "fv_checkpoint_bytes": [c_void_p, ctypes.POINTER(ctypes.c_size_t)],
    "fv_checkpoint_save": [c_void_p, c_void_p],
    "fv_checkpoint_load": [c_void_p, c_void_p],
    "fv_set_halo": [c_void_p, c_int, c_int],
    "fv_enqueue_stage": [c_void_p, c_void_p, c_int],
    "fv_halo_exchange": [c_void_p, c_int, c_int, c_int],
    "fv_reduce_dt": [c_void_p, c_int],
    "fv_halo_pack": [c_void_p, c_int, c_int, c_void_p],
    "fv_halo_unpack": [c_void_p, c_int, c_int, c_void_p],
    "fv_halo_strip_floats": [c_void_p, c_int, ctypes.POINTER(ctypes.c_longlong)],
    "fv_set_dt": [c_void_p, c_void_p],
    "fv_set_learned_hmin_values": [c_void_p, c_void_p],
    "fv_health": [c_void_p, c_void_p],
    "fv_diagnostics": [c_void_p, c_void_p],
}
_RESTYPES = {"fv_last_error": ctypes.c_char_p}


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it was never built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = _RESTYPES.get(name, c_int)
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(rc: int) -> int:
    if rc < 0:
        raise FvError(rc, lib().fv_last_error().decode())
    return rc


def _torch_stream() -> int:
    h = torch.cuda.current_stream().cuda_stream
    return h if h else CUDA_STREAM_LEGACY


def _ptr_loc(t: torch.Tensor):
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("state tensors must be contiguous float32")
    return ctypes.c_void_p(t.data_ptr()), (FV_DEVICE if t.is_cuda else FV_HOST)


class State:
    """Owner of an ``fv_state*`` handle."""

    def __init__(self, handle: int, eq: str, shape):
        self.handle = ctypes.c_void_p(handle)
        self.eq = eq
        self.shape = tuple(shape)   # (B, C, ny, nx)

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.fv_destroy_state(self.handle)
            self.handle = ctypes.c_void_p(0)

    @property
    def stream(self) -> int:
        out = c_void_p()
        _check(lib().fv_state_stream(self.handle, ctypes.byref(out)))
        return out.value or 0

    @property
    def device_ptr(self) -> int:
        out = c_void_p()
        _check(lib().fv_state_device_ptr(self.handle, ctypes.byref(out)))
        return out.value


def _grid(q: torch.Tensor, lx: float, ly: float) -> fv_grid:
    if q.dim() != 4:
        raise ValueError("q0 must be [B][C][ny][nx]")
    B, _, ny, nx = q.shape
    return fv_grid(nx, ny, B, lx, ly)


def swe_init(q0: torch.Tensor, g: float = 9.81, cfl: float = 0.5, dt_mode: str = "adaptive",
             dt_fixed: float = 0.0, lx: float = 1.0, ly: float = 1.0) -> State:
    q0 = q0.contiguous()
    if q0.shape[1] != 3:
        raise ValueError("SWE state has 3 variables")
    ptr, loc = _ptr_loc(q0)
    out = c_void_p()
    stream = c_void_p(_torch_stream()) if torch.cuda.is_available() else None
    _check(lib().swe_init(ctypes.byref(_grid(q0, lx, ly)),
                          ctypes.byref(fv_swe_params(g, cfl, DT_MODES[dt_mode], dt_fixed)),
                          ptr, loc, stream, ctypes.byref(out)))
    return State(out.value, "swe", q0.shape)


def euler_init(q0: torch.Tensor, gamma: float = 1.4, cfl: float = 0.5, dt_mode: str = "adaptive",
               dt_fixed: float = 0.0, lx: float = 1.0, ly: float = 1.0) -> State:
    q0 = q0.contiguous()
    if q0.shape[1] != 4:
        raise ValueError("Euler state has 4 variables")
    ptr, loc = _ptr_loc(q0)
    out = c_void_p()
    stream = c_void_p(_torch_stream()) if torch.cuda.is_available() else None
    _check(lib().euler_init(ctypes.byref(_grid(q0, lx, ly)),
                            ctypes.byref(fv_euler_params(gamma, cfl, DT_MODES[dt_mode], dt_fixed)),
                            ptr, loc, stream, ctypes.byref(out)))
    return State(out.value, "euler", q0.shape)


def sphere_init(q0: torch.Tensor, g: float, omega: float, cfl: float = 0.5, dt_mode: str = "adaptive",
                dt_fixed: float = 0.0) -> State:
    """Shallow water on the unit sphere: q0 [B][4][ny][nx] with nx = 2 ny,
    (h, hu, hv, hw) on the two-hemisphere grid (host or device tensor)."""
    q0 = q0.contiguous()
    if q0.dim() != 4 or q0.shape[1] != 4:
        raise ValueError("sphere state is [B][4][ny][nx]")
    B, _, ny, nx = q0.shape
    ptr, loc = _ptr_loc(q0)
    out = c_void_p()
    stream = c_void_p(_torch_stream()) if torch.cuda.is_available() else None
    _check(lib().sphere_init(nx, ny, B, ctypes.byref(fv_sphere_params(g, omega, cfl, DT_MODES[dt_mode], dt_fixed)),
                             ptr, loc, stream, ctypes.byref(out)))
    return State(out.value, "sphere", q0.shape)


def sphere_get_cells(s: State):
    """(unit cell centres [3][ny][nx], cell areas [ny][nx]) of a sphere state,
    as host numpy float32 arrays."""
    _, _, ny, nx = s.shape
    c = np.zeros((3, ny, nx), dtype=np.float32)
    a = np.zeros((ny, nx), dtype=np.float32)
    _check(lib().sphere_get_cells(s.handle, c.ctypes.data_as(c_void_p), a.ctypes.data_as(c_void_p), FV_HOST))
    return c, a


def fv_set_replay_dt(s: State, dts) -> None:
    a = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
    _check(lib().fv_set_replay_dt(s.handle, a.ctypes.data_as(c_void_p), a.size))


def _net_handle(net):
    return None if net is None else net.handle


def fv_step(s: State, net=None) -> None:
    _check(lib().fv_step(s.handle, _net_handle(net)))


def fv_enqueue_steps(s: State, nsteps: int, net=None) -> None:
    _check(lib().fv_enqueue_steps(s.handle, _net_handle(net), int(nsteps)))


def fv_sync(s: State) -> None:
    _check(lib().fv_sync(s.handle))


def fv_rollout(s: State, nsteps: int, net=None, t_end: float = 0.0, snap_every: int = 0,
               snaps_on_device: bool = True):
    """Run ``nsteps`` steps; returns ``(snaps or None, t_out[B])``."""
    B = s.shape[0]
    t_out = np.zeros(B, dtype=np.float64)
    snaps = None
    sptr, sloc = None, FV_DEVICE
    if snap_every:
        n = nsteps // snap_every
        dev = "cuda" if snaps_on_device else "cpu"
        snaps = torch.empty((n,) + s.shape, dtype=torch.float32, device=dev,
                            pin_memory=(not snaps_on_device))
        sptr, sloc = _ptr_loc(snaps)
    _check(lib().fv_rollout(s.handle, _net_handle(net), int(nsteps), float(t_end), sptr, sloc,
                            int(snap_every), t_out.ctypes.data_as(c_void_p)))
    return snaps, t_out


def fv_get_state(s: State, out: torch.Tensor | None = None, device: bool = True) -> torch.Tensor:
    if out is None:
        out = torch.empty(s.shape, dtype=torch.float32, device="cuda" if device else "cpu")
    ptr, loc = _ptr_loc(out)
    _check(lib().fv_get_state(s.handle, ptr, loc))
    return out


def fv_set_state(s: State, q: torch.Tensor) -> None:
    q = q.contiguous()
    ptr, loc = _ptr_loc(q)
    _check(lib().fv_set_state(s.handle, ptr, loc))


STAGE_VARIANTS = {"auto": 0, "tile": 1, "march": 2}


def fv_set_stage_variant(s: State, variant: str) -> None:
    _check(lib().fv_set_stage_variant(s.handle, STAGE_VARIANTS[variant]))


def fv_get_time(s: State):
    B = s.shape[0]
    t = np.zeros(B)
    dt = np.zeros(B)
    steps = np.zeros(B, dtype=np.int64)
    _check(lib().fv_get_time(s.handle, t.ctypes.data_as(c_void_p), dt.ctypes.data_as(c_void_p),
                             steps.ctypes.data_as(c_void_p)))
    return t, dt, steps


def fv_health(s: State) -> np.ndarray:
    f = np.zeros(s.shape[0], dtype=np.uint32)
    _check(lib().fv_health(s.handle, f.ctypes.data_as(c_void_p)))
    return f


def fv_diagnostics(s: State) -> np.ndarray:
    B, C = s.shape[:2]
    out = np.zeros((B, C + 1), dtype=np.float64)
    _check(lib().fv_diagnostics(s.handle, out.ctypes.data_as(c_void_p)))
    return out


def fv_checkpoint_save(s: State) -> bytes:
    """The state's checkpoint blob (header, control blocks, q^n)."""
    n = ctypes.c_size_t()
    _check(lib().fv_checkpoint_bytes(s.handle, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().fv_checkpoint_save(s.handle, ctypes.cast(buf, c_void_p)))
    return buf.raw


def fv_checkpoint_load(s: State, blob: bytes) -> None:
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().fv_checkpoint_load(s.handle, ctypes.cast(buf, c_void_p)))


# ---------------------------------------------------------------------------
# Subdomains of a block-decomposed grid (see decomp.py)
# ---------------------------------------------------------------------------

def fv_set_halo(s: State, hx: int, hy: int) -> None:
    _check(lib().fv_set_halo(s.handle, int(hx), int(hy)))


def fv_enqueue_stage(s: State, stage: int, net=None) -> None:
    _check(lib().fv_enqueue_stage(s.handle, _net_handle(net), int(stage)))


def fv_halo_exchange(subs_array, px: int, py: int, buf: int) -> None:
    """subs_array: a ctypes array of the px * py state handles (block order)."""
    _check(lib().fv_halo_exchange(ctypes.cast(subs_array, c_void_p), int(px), int(py), int(buf)))


def fv_reduce_dt(subs_array, n: int) -> None:
    _check(lib().fv_reduce_dt(ctypes.cast(subs_array, c_void_p), int(n)))


def fv_halo_strip_floats(s: State, side: int) -> int:
    n = ctypes.c_longlong()
    _check(lib().fv_halo_strip_floats(s.handle, int(side), ctypes.byref(n)))
    return n.value


def fv_halo_pack(s: State, buf: int, side: int, dst: torch.Tensor) -> None:
    _check(lib().fv_halo_pack(s.handle, int(buf), int(side), _dev(dst)))


def fv_halo_unpack(s: State, buf: int, side: int, src: torch.Tensor) -> None:
    _check(lib().fv_halo_unpack(s.handle, int(buf), int(side), _dev(src)))


def fv_set_dt(s: State, dt) -> None:
    a = np.ascontiguousarray(np.asarray(dt, dtype=np.float64))
    if a.size != s.shape[0]:
        raise ValueError("one dt per member")
    _check(lib().fv_set_dt(s.handle, a.ctypes.data_as(c_void_p)))


def fv_set_learned_hmin_values(s: State, hmin) -> None:
    a = np.ascontiguousarray(np.asarray(hmin, dtype=np.float64))
    if a.size != s.shape[0]:
        raise ValueError("one h_min per member")
    _check(lib().fv_set_learned_hmin_values(s.handle, a.ctypes.data_as(c_void_p)))


# ---------------------------------------------------------------------------
# Learned stencil network
# ---------------------------------------------------------------------------

FV_NET_PARAMS = 29796
FV_FACE_NET_PARAMS = 22860


class Net:
    """Owner of an ``fv_net*`` handle (a stencil or a face-state network)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)
        self.n_params = int(lib().fv_net_num_params(self.handle))
        self.kind = "face" if int(lib().fv_net_kind(self.handle)) == 1 else "stencil"

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.stencil_net_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)


def _host_params(params, n=FV_NET_PARAMS):
    a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
    if a.size != n:
        raise ValueError(f"expected {n} parameters, got {a.size}")
    return a


def stencil_net_create(params=None, mean=(0.0, 0.0, 0.0), std=(1.0, 1.0, 1.0)) -> Net:
    norm = np.ascontiguousarray(np.asarray(list(mean) + list(std), dtype=np.float32))
    out = c_void_p()
    p = None
    if params is not None:
        hp = _host_params(params)
        p = hp.ctypes.data_as(c_void_p)
    _check(lib().stencil_net_create(p, norm.ctypes.data_as(c_void_p), ctypes.byref(out)))
    return Net(out.value)


def stencil_net_set_params(net: Net, params) -> None:
    if isinstance(params, torch.Tensor) and params.is_cuda:
        t = params.contiguous().float()
        _check(lib().stencil_net_set_params(net.handle, c_void_p(t.data_ptr()), FV_DEVICE))
        return
    hp = _host_params(params, net.n_params)
    _check(lib().stencil_net_set_params(net.handle, hp.ctypes.data_as(c_void_p), FV_HOST))


def stencil_net_get_params(net: Net, out: torch.Tensor | None = None):
    """Parameters as a numpy array, or into the given CUDA tensor."""
    if out is not None:
        _check(lib().stencil_net_get_params(net.handle, _dev(out), FV_DEVICE))
        return out
    host = np.zeros(net.n_params, dtype=np.float32)
    _check(lib().stencil_net_get_params(net.handle, host.ctypes.data_as(c_void_p), FV_HOST))
    return host


def stencil_net_forward(net: Net, q: torch.Tensor, raw: bool = False) -> torch.Tensor:
    """Normalised coefficients (or raw outputs) [B][36][ny][nx] for q on the GPU."""
    q = q.contiguous()
    if not q.is_cuda or q.dtype != torch.float32 or q.dim() != 4 or q.shape[1] != 3:
        raise ValueError("q must be a CUDA float32 tensor [B][3][ny][nx]")
    B, _, ny, nx = q.shape
    out = torch.empty((B, 36, ny, nx), dtype=torch.float32, device=q.device)
    _check(lib().stencil_net_forward(net.handle, c_void_p(q.data_ptr()), B, ny, nx,
                                     c_void_p(out.data_ptr()), int(raw),
                                     c_void_p(_torch_stream())))
    return out


def face_net_create(params=None, mean=(0.0, 0.0, 0.0), std=(1.0, 1.0, 1.0)) -> Net:
    """Face-state network (Section 2.5.3, third approach); params host
    [FV_FACE_NET_PARAMS] or None (zeros)."""
    norm = np.ascontiguousarray(np.asarray(list(mean) + list(std), dtype=np.float32))
    out = c_void_p()
    p = None
    if params is not None:
        hp = _host_params(params, FV_FACE_NET_PARAMS)
        p = hp.ctypes.data_as(c_void_p)
    _check(lib().face_net_create(p, norm.ctypes.data_as(c_void_p), ctypes.byref(out)))
    return Net(out.value)


def face_net_forward(net: Net, q: torch.Tensor, raw: bool = False) -> torch.Tensor:
    """Side states (or raw outputs) [B][12][ny][nx] for q on the GPU."""
    q = q.contiguous()
    if not q.is_cuda or q.dtype != torch.float32 or q.dim() != 4 or q.shape[1] != 3:
        raise ValueError("q must be a CUDA float32 tensor [B][3][ny][nx]")
    B, _, ny, nx = q.shape
    out = torch.empty((B, 12, ny, nx), dtype=torch.float32, device=q.device)
    _check(lib().face_net_forward(net.handle, c_void_p(q.data_ptr()), B, ny, nx,
                                  c_void_p(out.data_ptr()), int(raw), c_void_p(_torch_stream())))
    return out


def net_backward(net: Net, q: torch.Tensor, dout: torch.Tensor, want_dq: bool = True,
                 dparams: torch.Tensor | None = None, dq: torch.Tensor | None = None):
    """Vector-Jacobian product of the network's forward at q: dout is the
    cotangent of its output ([B][36][ny][nx] coefficients of a stencil
    network, [B][12][ny][nx] side states of a face-state network).  The
    gradients are added to ``dparams`` [n_params] and ``dq`` [B][3][ny][nx]
    (zero-filled when not given); returns (dparams, dq or None) on the GPU."""
    q = q.contiguous()
    dout = dout.contiguous()
    B, _, ny, nx = q.shape
    if dparams is None:
        dparams = torch.zeros(net.n_params, dtype=torch.float32, device=q.device)
    if want_dq and dq is None:
        dq = torch.zeros_like(q)
    if not want_dq:
        dq = None
    fn = lib().face_net_backward if net.kind == "face" else lib().stencil_net_backward
    _check(fn(net.handle, _dev(q), B, ny, nx, _dev(dout), _dev(dq) if want_dq else None, _dev(dparams),
              c_void_p(_torch_stream())))
    return dparams, dq


FLUXES = {"hll": 0, "rusanov": 1, "lf": 2, "roe": 3, "hlle": 4, "hllc": 5}


def fv_set_scheme(s: State, flux: str = "hll", rk: int = 2) -> None:
    """Numerical flux ("hll", "rusanov", "lf", "roe", "hlle", "hllc") and
    integrator (2: SSP-RK2, 3: SSP-RK3) of the plain step."""
    _check(lib().fv_set_scheme(s.handle, FLUXES[flux], int(rk)))


BOUNDARIES = {"periodic": 0, "wall": 1}


def fv_set_boundary(s: State, bc: str) -> None:
    """"periodic" (default) or "wall" (reflecting) on all four sides."""
    _check(lib().fv_set_boundary(s.handle, BOUNDARIES[bc]))


def fv_set_bathymetry(s: State, z) -> None:
    """Shallow-water bed z [ny][nx] at the cell centres (a torch tensor on
    the host or the device, or None for a flat bed)."""
    if z is None:
        _check(lib().fv_set_bathymetry(s.handle, None, FV_HOST))
        return
    zt = z.detach().to(torch.float32).contiguous()
    if tuple(zt.shape) != tuple(s.shape[-2:]):
        raise ValueError(f"bed shape {tuple(zt.shape)} != grid {tuple(s.shape[-2:])}")
    loc = FV_DEVICE if zt.is_cuda else FV_HOST
    _check(lib().fv_set_bathymetry(s.handle, c_void_p(zt.data_ptr()), loc))


LEARNED_VARIANTS = {"auto": 0, "fused": 1, "two_pass": 2}


def fv_set_learned_variant(s: State, variant: str) -> None:
    """Learned step implementation: "auto", "fused" (one persistent kernel
    per stage, nx a multiple of 128 up to 1024) or "two_pass" (CNN to device
    memory, then the stage kernel)."""
    _check(lib().fv_set_learned_variant(s.handle, LEARNED_VARIANTS[variant]))


def fv_set_learned_hmin(s: State, hmin_frac: float) -> None:
    _check(lib().fv_set_learned_hmin(s.handle, float(hmin_frac)))


# ---------------------------------------------------------------------------
# Training
# ---------------------------------------------------------------------------

class Tape:
    """Owner of an ``fv_tape*`` (keeps its network alive)."""

    def __init__(self, handle: int, net: Net, shape, T: int):
        self.handle = ctypes.c_void_p(handle)
        self.net = net
        self.shape = tuple(shape)   # (B, 3, ny, nx)
        self.T = T
        self.recorded = 0           # forward passes recorded so far

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.fv_tape_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)


def fv_tape_create(net: Net, B: int, ny: int, nx: int, T: int, dt: float, g: float = 9.81,
                   hmin_frac: float = 1e-3) -> Tape:
    out = c_void_p()
    _check(lib().fv_tape_create(net.handle, B, ny, nx, T, dt, g, hmin_frac, ctypes.byref(out)))
    return Tape(out.value, net, (B, 3, ny, nx), T)


def _dev(t: torch.Tensor) -> c_void_p:
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA float32 tensor")
    return c_void_p(t.data_ptr())


def fv_tape_forward(tape: Tape, q0: torch.Tensor, want_snaps: bool = True):
    torch.cuda.current_stream().synchronize()
    snaps = torch.empty((tape.T,) + tape.shape, dtype=torch.float32, device="cuda") if want_snaps else None
    tape.recorded += 1
    _check(lib().fv_tape_forward(tape.handle, _dev(q0.contiguous()), _dev(snaps) if want_snaps else None))
    return snaps


def fv_tape_loss(tape: Tape, targets: torch.Tensor, scale) -> float:
    torch.cuda.current_stream().synchronize()
    sc = np.ascontiguousarray(np.asarray(scale, dtype=np.float32))
    out = c_double()
    _check(lib().fv_tape_loss(tape.handle, _dev(targets.contiguous()), sc.ctypes.data_as(c_void_p),
                              ctypes.byref(out)))
    return out.value


def fv_tape_backward(tape: Tape, dparams: torch.Tensor, dsnaps: torch.Tensor | None = None,
                     want_dq0: bool = False):
    torch.cuda.current_stream().synchronize()
    dq0 = torch.empty(tape.shape, dtype=torch.float32, device="cuda") if want_dq0 else None
    _check(lib().fv_tape_backward(tape.handle, _dev(dsnaps.contiguous()) if dsnaps is not None else None,
                                  _dev(dparams), _dev(dq0) if want_dq0 else None))
    return dq0


class TapeRollout(torch.autograd.Function):
    """The learned rollout as a differentiable torch function:
    (params, q0) -> snaps [T][B][3][ny][nx], the states after steps 1..T.

    forward sets the network's parameters and records the tape
    (fv_tape_forward); backward is the library's hand-written adjoint
    (fv_tape_backward) with the incoming cotangent of the snapshots.  A tape
    holds one recorded window, so a backward must follow its own forward
    before the tape records another one (checked)."""

    @staticmethod
    def forward(ctx, params, q0, tape):
        stencil_net_set_params(tape.net, params.detach())
        snaps = fv_tape_forward(tape, q0.detach().contiguous())
        ctx.tape = tape
        ctx.generation = tape.recorded
        return snaps

    @staticmethod
    def backward(ctx, dsnaps):
        tape = ctx.tape
        if tape.recorded != ctx.generation:
            raise RuntimeError("the tape has recorded another rollout since this forward")
        dparams = torch.zeros(tape.net.n_params, dtype=torch.float32, device="cuda")
        dq0 = fv_tape_backward(tape, dparams, dsnaps.float().contiguous(), want_dq0=True)
        return dparams, dq0, None


def tape_rollout(tape: Tape, params: torch.Tensor, q0: torch.Tensor) -> torch.Tensor:
    """Differentiable learned rollout (see TapeRollout): params [n_params]
    and q0 [B][3][ny][nx], CUDA float32."""
    return TapeRollout.apply(params, q0, tape)


def stencil_net_adam_step(net: Net, grad: torch.Tensor, step: int, lr: float = 1e-3,
                          b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> None:
    torch.cuda.current_stream().synchronize()
    _check(lib().stencil_net_adam_step(net.handle, _dev(grad), int(step), lr, b1, b2, eps))


def fv_coarsen(q: torch.Tensor, factor: int) -> torch.Tensor:
    """Block means of factor x factor cells of a CUDA tensor [..., ny, nx]."""
    q = q.contiguous()
    ny, nx = q.shape[-2:]
    planes = int(np.prod(q.shape[:-2])) if q.dim() > 2 else 1
    out = torch.empty(q.shape[:-2] + (ny // factor, nx // factor), dtype=torch.float32, device=q.device)
    _check(lib().fv_coarsen(_dev(q), planes, ny, nx, factor, _dev(out), c_void_p(_torch_stream())))
    return out


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------

class fv_request(ctypes.Structure):
    _fields_ = [("eq", c_int), ("learned", c_int), ("nx", c_int), ("ny", c_int), ("nsteps", c_long),
                ("cfl", c_double), ("q0", c_void_p)]


class Server:
    """Owner of an ``fv_server*`` (keeps its network alive)."""

    def __init__(self, handle: int, net=None):
        self.handle = ctypes.c_void_p(handle)
        self.net = net
        self.shapes = {}

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.fv_server_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)


def fv_server_create(hbm_budget_bytes: int, max_slots: int, net: Net | None = None) -> Server:
    out = c_void_p()
    _check(lib().fv_server_create(int(hbm_budget_bytes), int(max_slots),
                                  net.handle if net is not None else None, ctypes.byref(out)))
    return Server(out.value, net)


def submit(server: Server, q0, eq: str = "swe", nsteps: int = 100, learned: bool = False,
           cfl: float = 0.5) -> int:
    """Queue a request for q0 (host [C][ny][nx]); returns its ticket."""
    a = np.ascontiguousarray(np.asarray(q0, dtype=np.float32))
    C, ny, nx = a.shape
    r = fv_request(0 if eq == "swe" else 1, int(learned), nx, ny, int(nsteps), float(cfl),
                   a.ctypes.data_as(c_void_p))
    t = ctypes.c_ulonglong()
    _check(lib().fv_submit(server.handle, ctypes.byref(r), ctypes.byref(t)))
    server.shapes[t.value] = a.shape
    return t.value


def poll(server: Server, ticket: int):
    """None while pending, else (final state [C][ny][nx], latency in s)."""
    shape = server.shapes[ticket]
    out = np.empty(shape, dtype=np.float32)
    lat = c_double()
    rc = lib().fv_poll(server.handle, ctypes.c_ulonglong(ticket), out.ctypes.data_as(c_void_p),
                       ctypes.byref(lat))
    if rc == FV_PENDING:
        return None
    del server.shapes[ticket]
    _check(rc)
    return out, lat.value


def fv_server_stats(server: Server):
    """(active, pending, device bytes reserved, learned requests that fell back)."""
    a, p, u, f = c_int(), c_int(), ctypes.c_size_t(), ctypes.c_longlong()
    _check(lib().fv_server_stats(server.handle, ctypes.byref(a), ctypes.byref(p), ctypes.byref(u),
                                 ctypes.byref(f)))
    return a.value, p.value, u.value, f.value
