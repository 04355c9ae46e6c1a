"""Thin ctypes binding of liblj.so (C ABI in include/lj.h).

The functions carry the C names and do argument marshalling only: they check
dtypes, shapes and devices of torch tensors and pass raw pointers.  Every
step of the MD path runs in the library's CUDA kernels; there is no CPU
fallback.  If the library has not been built, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblj.so")

LJ_OK, LJ_EINVAL, LJ_EBOX, LJ_ECUDA, LJ_ENONFINITE, LJ_ETIMEOUT, LJ_EOVERFLOW, LJ_ENOMEM = range(8)
LJ_SHIFT_NONE, LJ_SHIFT_ENERGY, LJ_SHIFT_FORCE = 0, 1, 2
LJ_PREC_MIXED, LJ_PREC_FP64 = 0, 1
LJ_FLAG_RUN_STAGED = 1
LJ_FLAG_RUN_DIRECT = 2

_PREC = {"mixed": LJ_PREC_MIXED, "fp64": LJ_PREC_FP64, LJ_PREC_MIXED: LJ_PREC_MIXED, LJ_PREC_FP64: LJ_PREC_FP64}


class lj_params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("box", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("rc", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("shift_mode", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("cell_subdiv", ctypes.c_int32),
        ("flags", ctypes.c_int32),
    ]


def make_params(n: int, box: float, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5,
                dt: float = 0.005, mass: float = 1.0, shift_mode: int = LJ_SHIFT_ENERGY,
                precision="mixed", cell_subdiv: int = 1, flags: int = 0) -> lj_params:
    return lj_params(int(n), float(box), float(eps), float(sigma), float(rc), float(dt), float(mass),
                     int(shift_mode), _PREC[precision], int(cell_subdiv), int(flags))


class LJError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {lj_strerror(code)} (status {code})")


_lock = threading.Lock()
_lib = None

# Every entry point of include/lj.h with its ctypes signature.
_P = ctypes.c_void_p
_SIGS = {
    "lj_version": ([], ctypes.c_int),
    "lj_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "lj_grid": ([ctypes.POINTER(lj_params), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "lj_create": ([ctypes.POINTER(_P), ctypes.POINTER(lj_params), _P], ctypes.c_int),
    "lj_destroy": ([_P], None),
    "lj_bin": ([_P, _P], ctypes.c_int),
    "lj_get_cells": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "lj_forces_n2": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "lj_srand48_state": ([ctypes.c_int64], ctypes.c_uint64),
    "lj_set_skin": ([_P, ctypes.c_double, ctypes.c_int32], ctypes.c_int),
    "lj_set_graph": ([_P, ctypes.c_int32], ctypes.c_int),
    "lj_set_deterministic": ([_P, ctypes.c_int32], ctypes.c_int),
    "lj_wait_selftest": ([_P], ctypes.c_int),
    "lj_skin_stats": ([_P, _P, _P], ctypes.c_int),
    "lj_rand48_jump": ([ctypes.c_int64, _P, _P], ctypes.c_int),
    "lj_rand48_seed": ([_P, ctypes.c_int64, ctypes.c_uint64, _P], ctypes.c_int),
    "lj_rand48_lrand": ([_P, ctypes.c_int64, ctypes.c_int64, _P, _P], ctypes.c_int),
    "lj_rand48_drand": ([_P, ctypes.c_int64, ctypes.c_int64, _P, _P], ctypes.c_int),
    "lj_langevin_seed": ([_P, ctypes.c_int64], ctypes.c_int),
    "lj_langevin_step": ([_P, _P, _P, _P, ctypes.c_int32, ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "lj_get_rng_state": ([_P, _P], ctypes.c_int),
    "lj_set_rng_state": ([_P, _P], ctypes.c_int),
    "lj_forces": ([_P, _P, _P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "lj_step": ([_P, _P, _P, _P, ctypes.c_int32], ctypes.c_int),
    "lj_step_host": ([_P, _P, _P, _P, ctypes.c_int32], ctypes.c_int),
    "lj_energy": ([_P, _P, _P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "lj_observables": ([_P, _P, _P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "lj_check": ([_P], ctypes.c_int),
    "lj_set_params": ([_P, ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "lj_set_tuning": ([_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "lj_batch_create": ([ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(lj_params), _P], ctypes.c_int),
    "lj_batch_destroy": ([_P], None),
    "lj_batch_info": ([_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "lj_batch_set_tuning": ([_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "lj_batch_set_kernel": ([_P, ctypes.c_int32], ctypes.c_int),
    "lj_batch_forces": ([_P, _P, _P, ctypes.c_int32], ctypes.c_int),
    "lj_batch_step": ([_P, _P, _P, _P, ctypes.c_int32], ctypes.c_int),
    "lj_batch_energy": ([_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "lj_batch_relax": ([_P, _P, _P, ctypes.c_int32, ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "lj_batch_check": ([_P], ctypes.c_int),
    "lj_batch_launches": ([_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "lj_forces_vjp": ([_P, _P, _P, ctypes.c_double, _P, _P], ctypes.c_int),
    "lj_vv_adjoint_step": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "lj_forces_static": ([ctypes.POINTER(lj_params), _P, _P, _P], ctypes.c_int),
    "lj_measure_peak": ([ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "lj_set_timing": ([_P, ctypes.c_int32], ctypes.c_int),
    "lj_read_timing": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
}


def load() -> ctypes.CDLL:
    """Load liblj.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                               "(the CUDA library is required: there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _ck(code: int, where: str) -> None:
    if code != LJ_OK:
        raise LJError(code, where)


def lj_version() -> int:
    return load().lj_version()


def lj_strerror(code: int) -> str:
    return load().lj_strerror(int(code)).decode()


def lj_grid(params: lj_params) -> int:
    nc = ctypes.c_int32()
    _ck(load().lj_grid(ctypes.byref(params), ctypes.byref(nc)), "lj_grid")
    return nc.value


def _stream_ptr(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def _dev(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """Owns an lj_ctx*; ``params`` and ``nc`` are kept for marshalling."""

    def __init__(self, params: lj_params, stream=None):
        self.params = params
        self.nc = lj_grid(params)
        self.stream = stream
        h = ctypes.c_void_p()
        _ck(load().lj_create(ctypes.byref(h), ctypes.byref(params), _stream_ptr(stream)), "lj_create")
        self.handle = h

    @property
    def n(self) -> int:
        return int(self.params.n)

    @property
    def force_dtype(self):
        import torch
        return torch.float64 if self.params.precision == LJ_PREC_FP64 else torch.float32

    def close(self) -> None:
        if self.handle:
            load().lj_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lj_create(params: lj_params, stream=None) -> Context:
    return Context(params, stream)


def lj_destroy(ctx: Context) -> None:
    ctx.close()


def lj_bin(ctx: Context, x) -> None:
    import torch
    _ck(load().lj_bin(ctx.handle, _dev(x, torch.float64, (ctx.n, 3), "x")), "lj_bin")


def lj_get_cells(ctx: Context, cell_of=None, count=None, start=None, perm=None) -> None:
    import torch
    ncell = ctx.nc ** 3
    a = [None if cell_of is None else _dev(cell_of, torch.int32, (ctx.n,), "cell_of"),
         None if count is None else _dev(count, torch.int32, (ncell,), "count"),
         None if start is None else _dev(start, torch.int32, (ncell + 1,), "start"),
         None if perm is None else _dev(perm, torch.int32, (ctx.n,), "perm")]
    _ck(load().lj_get_cells(ctx.handle, *a), "lj_get_cells")


def lj_forces(ctx: Context, x, f, energy: bool = False):
    """Forces into f (n, 4); with energy=True returns (e_pot, virial)."""
    import torch
    xp = _dev(x, torch.float64, (ctx.n, 3), "x")
    fp = _dev(f, ctx.force_dtype, (ctx.n, 4), "f")
    if energy:
        e = ctypes.c_double()
        w = ctypes.c_double()
        _ck(load().lj_forces(ctx.handle, xp, fp, ctypes.byref(e), ctypes.byref(w)), "lj_forces")
        return e.value, w.value
    _ck(load().lj_forces(ctx.handle, xp, fp, None, None), "lj_forces")
    return None


def lj_forces_n2(ctx: Context, x, f, energy: bool = False):
    """All-pairs forces (no cells) into f (n, 4); with energy=True returns
    (e_pot, virial)."""
    import torch
    xp = _dev(x, torch.float64, (ctx.n, 3), "x")
    fp = _dev(f, ctx.force_dtype, (ctx.n, 4), "f")
    if energy:
        e = ctypes.c_double()
        w = ctypes.c_double()
        _ck(load().lj_forces_n2(ctx.handle, xp, fp, ctypes.byref(e), ctypes.byref(w)), "lj_forces_n2")
        return e.value, w.value
    _ck(load().lj_forces_n2(ctx.handle, xp, fp, None, None), "lj_forces_n2")
    return None


def lj_set_skin(ctx: Context, skin: float, max_interval: int = 0) -> None:
    """Cell lists with a skin: cells >= (rc + skin) wide, rebuilt only when
    some particle has moved skin/2 (or every max_interval steps)."""
    import math
    _ck(load().lj_set_skin(ctx.handle, float(skin), int(max_interval)), "lj_set_skin")
    k = ctx.params.cell_subdiv or 1
    ctx.nc = int(math.floor((k * ctx.params.box) / (ctx.params.rc + float(skin))))


def lj_wait_selftest(ctx: Context) -> int:
    """Run one unsatisfiable bounded device wait; returns the status lj_check
    reports afterwards (LJ_ETIMEOUT when the bound works)."""
    return int(load().lj_wait_selftest(ctx.handle))


def lj_set_deterministic(ctx: Context, enable: bool = True) -> None:
    """Sort each cell's particles by index at every binning."""
    _ck(load().lj_set_deterministic(ctx.handle, 1 if enable else 0), "lj_set_deterministic")


def lj_set_graph(ctx: Context, enable: bool = True) -> None:
    """Replay the middle steps of lj_step from one captured CUDA graph."""
    _ck(load().lj_set_graph(ctx.handle, 1 if enable else 0), "lj_set_graph")


def lj_skin_stats(ctx: Context) -> tuple[int, int]:
    r = ctypes.c_int64()
    n = ctypes.c_int64()
    _ck(load().lj_skin_stats(ctx.handle, ctypes.byref(r), ctypes.byref(n)), "lj_skin_stats")
    return r.value, n.value


def lj_srand48_state(seed: int) -> int:
    return int(load().lj_srand48_state(int(seed)))


def lj_rand48_jump(m: int) -> tuple[int, int]:
    A = ctypes.c_uint64()
    C = ctypes.c_uint64()
    _ck(load().lj_rand48_jump(int(m), ctypes.byref(A), ctypes.byref(C)), "lj_rand48_jump")
    return int(A.value), int(C.value)


def _state(state):
    import torch
    if not (isinstance(state, torch.Tensor) and state.is_cuda and state.dtype == torch.int64
            and state.is_contiguous() and state.dim() == 1):
        raise TypeError("state must be a contiguous 1-D CUDA int64 tensor (uint64 bit patterns)")
    return ctypes.c_void_p(state.data_ptr()), state.numel()


def lj_rand48_seed(state, x0: int, stream=None) -> None:
    """state[i] = x_{i+1} of the series from x0 (state: CUDA int64 tensor)."""
    p, S = _state(state)
    _ck(load().lj_rand48_seed(p, S, ctypes.c_uint64(int(x0)), _stream_ptr(stream)), "lj_rand48_seed")


def lj_rand48_lrand(state, R: int, out=None, stream=None):
    """R rounds of lrand48 values from every stream: out (R * S,) int32."""
    import torch
    p, S = _state(state)
    if out is None:
        out = torch.empty(int(R) * S, dtype=torch.int32, device=state.device)
    o = _dev(out, torch.int32, (int(R) * S,), "out")
    _ck(load().lj_rand48_lrand(p, S, int(R), o, _stream_ptr(stream)), "lj_rand48_lrand")
    return out


def lj_rand48_drand(state, R: int, out=None, stream=None):
    """R rounds of drand48 values from every stream: out (R * S,) float64."""
    import torch
    p, S = _state(state)
    if out is None:
        out = torch.empty(int(R) * S, dtype=torch.float64, device=state.device)
    o = _dev(out, torch.float64, (int(R) * S,), "out")
    _ck(load().lj_rand48_drand(p, S, int(R), o, _stream_ptr(stream)), "lj_rand48_drand")
    return out


def lj_langevin_seed(ctx: Context, seed: int) -> None:
    _ck(load().lj_langevin_seed(ctx.handle, int(seed)), "lj_langevin_seed")


def lj_langevin_step(ctx: Context, x, v, f, nsteps: int, gamma: float, kT: float) -> None:
    import torch
    _ck(load().lj_langevin_step(ctx.handle, _dev(x, torch.float64, (ctx.n, 3), "x"),
                                _dev(v, torch.float64, (ctx.n, 3), "v"), _dev(f, ctx.force_dtype, (ctx.n, 4), "f"),
                                int(nsteps), float(gamma), float(kT)), "lj_langevin_step")


def lj_get_rng_state(ctx: Context, state=None):
    """The thermostat's n stream states (CUDA int64 tensor of uint64 bit
    patterns, each below 2^48); raises LJ_EINVAL before it was seeded."""
    import torch
    if state is None:
        state = torch.empty(ctx.n, dtype=torch.int64, device=torch.device("cuda", torch.cuda.current_device()))
    _ck(load().lj_get_rng_state(ctx.handle, _dev(state, torch.int64, (ctx.n,), "state")), "lj_get_rng_state")
    return state


def lj_set_rng_state(ctx: Context, state) -> None:
    """Load n stream states (CUDA int64 tensor, as lj_get_rng_state gives)."""
    import torch
    _ck(load().lj_set_rng_state(ctx.handle, _dev(state, torch.int64, (ctx.n,), "state")), "lj_set_rng_state")


def lj_step(ctx: Context, x, v, f, nsteps: int) -> None:
    import torch
    _ck(load().lj_step(ctx.handle, _dev(x, torch.float64, (ctx.n, 3), "x"),
                       _dev(v, torch.float64, (ctx.n, 3), "v"),
                       _dev(f, ctx.force_dtype, (ctx.n, 4), "f"), int(nsteps)), "lj_step")


def _host(a, dtype, shape, name):
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != dtype or tuple(a.shape) != tuple(shape) or not a.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU {dtype} tensor of shape {tuple(shape)}")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        npd = np.float64 if dtype == torch.float64 else np.float32
        if a.dtype != npd or a.shape != tuple(shape) or not a.flags.c_contiguous:
            raise ValueError(f"{name} must be a C-contiguous {npd.__name__} array of shape {tuple(shape)}")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"{name} must be a CPU tensor or numpy array")


def lj_step_host(ctx: Context, x, v, f, nsteps: int) -> None:
    """lj_step on host arrays (numpy or CPU tensors, pinned or not)."""
    import torch
    _ck(load().lj_step_host(ctx.handle, _host(x, torch.float64, (ctx.n, 3), "x"),
                            _host(v, torch.float64, (ctx.n, 3), "v"),
                            _host(f, ctx.force_dtype, (ctx.n, 4), "f"), int(nsteps)), "lj_step_host")


def lj_energy(ctx: Context, x, v) -> tuple[float, float, float]:
    """(kinetic, potential, total) energy, FP64."""
    import torch
    out = (ctypes.c_double * 3)()
    _ck(load().lj_energy(ctx.handle, _dev(x, torch.float64, (ctx.n, 3), "x"),
                         _dev(v, torch.float64, (ctx.n, 3), "v"), out), "lj_energy")
    return out[0], out[1], out[2]


def lj_observables(ctx: Context, x, v) -> dict:
    """E_kin, E_pot, E_tot, virial W, temperature T and virial pressure P
    (FP64; T and P formed on the device)."""
    import torch
    out = (ctypes.c_double * 6)()
    _ck(load().lj_observables(ctx.handle, _dev(x, torch.float64, (ctx.n, 3), "x"),
                              _dev(v, torch.float64, (ctx.n, 3), "v"), out), "lj_observables")
    keys = ("e_kin", "e_pot", "e_tot", "virial", "T", "P")
    return {k: out[i] for i, k in enumerate(keys)}


def lj_set_params(ctx: Context, eps: float, sigma: float) -> None:
    _ck(load().lj_set_params(ctx.handle, float(eps), float(sigma)), "lj_set_params")
    ctx.params.eps = float(eps)
    ctx.params.sigma = float(sigma)


def lj_forces_vjp(ctx: Context, x, g, scale: float, dx, dparam) -> None:
    """dx += scale dL/dx and dparam += scale (dL/deps, dL/dsigma) for g = dL/dF."""
    import torch
    _ck(load().lj_forces_vjp(ctx.handle, _dev(x, torch.float64, (ctx.n, 3), "x"),
                             _dev(g, torch.float64, (ctx.n, 3), "g"), float(scale),
                             _dev(dx, torch.float64, (ctx.n, 3), "dx"),
                             _dev(dparam, torch.float64, (2,), "dparam")), "lj_forces_vjp")


def lj_vv_adjoint_step(ctx: Context, x_n, x_n1, lam_x, lam_v, dparam) -> None:
    """One velocity-Verlet adjoint step (see include/lj.h), in place."""
    import torch
    _ck(load().lj_vv_adjoint_step(ctx.handle, _dev(x_n, torch.float64, (ctx.n, 3), "x_n"),
                                  _dev(x_n1, torch.float64, (ctx.n, 3), "x_n1"),
                                  _dev(lam_x, torch.float64, (ctx.n, 3), "lam_x"),
                                  _dev(lam_v, torch.float64, (ctx.n, 3), "lam_v"),
                                  _dev(dparam, torch.float64, (2,), "dparam")), "lj_vv_adjoint_step")


def lj_set_tuning(ctx: Context, kernel: int, group_width: int = 0, cells_per_grab: int = 4) -> None:
    """Force kernel of a context: 0 warp-per-cell with fused update (mixed),
    1 run-staged, 2 run-direct, 3 warp-per-cell with separate update (mixed);
    group_width 0 (compiled default), -1 (per cell), 2, 4, 8, 16 or 32;
    cells_per_grab 0 (static striding) or 1..1024."""
    _ck(load().lj_set_tuning(ctx.handle, int(kernel), int(group_width), int(cells_per_grab)), "lj_set_tuning")


class Batch:
    """Owns an lj_batch* (see include/lj.h) and its device state.

    ``xs``, ``vs``: lists of per-replica (n_r, 3) arrays; ``boxes``: per-replica
    box sides.  State is concatenated: x, v (sum n, 3) float64, f (sum n, 4)
    float32 CUDA tensors; ``offsets[r]:offsets[r+1]`` is replica r."""

    def __init__(self, xs, vs, boxes, *, eps=1.0, sigma=1.0, rc=2.5, dt=0.005, mass=1.0,
                 shift_mode=LJ_SHIFT_ENERGY, cell_subdiv=1, stream=None):
        import torch
        ns = [int(np.asarray(a).shape[0]) for a in xs]
        self.nrep = len(ns)
        self.offsets = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        self.boxes = [float(b) for b in boxes]
        self.x = torch.as_tensor(np.concatenate([np.asarray(a, np.float64) for a in xs])).cuda().contiguous()
        if vs is None:
            self.v = torch.zeros_like(self.x)
        else:
            self.v = torch.as_tensor(np.concatenate([np.asarray(a, np.float64) for a in vs])).cuda().contiguous()
        self.f = torch.zeros((self.x.shape[0], 4), dtype=torch.float32, device="cuda")
        self.params = make_params(0, 1.0, eps, sigma, rc, dt, mass, shift_mode, "mixed", cell_subdiv)
        self.cell_subdiv = int(cell_subdiv) or 1
        n_arr = (ctypes.c_int64 * self.nrep)(*ns)
        b_arr = (ctypes.c_double * self.nrep)(*self.boxes)
        h = ctypes.c_void_p()
        _ck(load().lj_batch_create(ctypes.byref(h), self.nrep, n_arr, b_arr, ctypes.byref(self.params),
                                   _stream_ptr(stream)), "lj_batch_create")
        self.handle = h
        self._forces_valid = False
        self.kernel = 3

    @property
    def ntot(self) -> int:
        return int(self.offsets[-1])

    def info(self):
        nt, nc = ctypes.c_int64(), ctypes.c_int64()
        g, cap = ctypes.c_int32(), ctypes.c_int32()
        _ck(load().lj_batch_info(self.handle, ctypes.byref(nt), ctypes.byref(nc), ctypes.byref(g),
                                 ctypes.byref(cap)), "lj_batch_info")
        return {"ntot": nt.value, "ncell": nc.value, "grid": g.value, "cap": cap.value}

    def set_tuning(self, cells_per_grab: int = 4, use_graph: bool = True, group_width: int = 0) -> None:
        _ck(load().lj_batch_set_tuning(self.handle, int(cells_per_grab), 1 if use_graph else 0, int(group_width)),
            "lj_batch_set_tuning")

    def set_kernel(self, kernel: int) -> None:
        """3: the 27-cell code (default); 7: each pair once (cell subdivision 1)."""
        _ck(load().lj_batch_set_kernel(self.handle, int(kernel)), "lj_batch_set_kernel")
        self.kernel = int(kernel)

    def forces(self, energy: bool = False) -> None:
        _ck(load().lj_batch_forces(self.handle, ctypes.c_void_p(self.x.data_ptr()),
                                   ctypes.c_void_p(self.f.data_ptr()), 1 if energy else 0), "lj_batch_forces")
        self._forces_valid = True

    def step(self, nsteps: int) -> None:
        if not self._forces_valid:
            self.forces()
        _ck(load().lj_batch_step(self.handle, ctypes.c_void_p(self.x.data_ptr()),
                                 ctypes.c_void_p(self.v.data_ptr()), ctypes.c_void_p(self.f.data_ptr()),
                                 int(nsteps)), "lj_batch_step")

    def energy(self) -> np.ndarray:
        out = (ctypes.c_double * (3 * self.nrep))()
        _ck(load().lj_batch_energy(self.handle, ctypes.c_void_p(self.x.data_ptr()),
                                   ctypes.c_void_p(self.v.data_ptr()), ctypes.c_void_p(self.f.data_ptr()), out),
            "lj_batch_energy")
        self._forces_valid = True
        return np.array(out).reshape(self.nrep, 3)

    def relax(self, nsteps: int, alpha: float, max_disp: float) -> None:
        _ck(load().lj_batch_relax(self.handle, ctypes.c_void_p(self.x.data_ptr()),
                                  ctypes.c_void_p(self.f.data_ptr()), int(nsteps), float(alpha),
                                  float(max_disp)), "lj_batch_relax")
        self._forces_valid = True

    def check(self) -> None:
        _ck(load().lj_batch_check(self.handle), "lj_batch_check")

    def launches(self):
        n, g = ctypes.c_int64(), ctypes.c_int32()
        _ck(load().lj_batch_launches(self.handle, ctypes.byref(n), ctypes.byref(g)), "lj_batch_launches")
        return n.value, bool(g.value)

    def replica(self, t, r: int):
        return t[int(self.offsets[r]):int(self.offsets[r + 1])]

    def close(self) -> None:
        if self.handle:
            load().lj_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


LJ_STATIC_MAX_N = 32768
LJ_STATIC_MAX_CELLS = 32768


def lj_forces_static(params: lj_params, x, f, stream=None) -> None:
    """Forces into f with no device allocation (fixed static scratch inside
    the library; see include/lj.h): for callers that cannot allocate.  n and
    cells per side are limited (LJ_STATIC_MAX_N, LJ_STATIC_MAX_CELLS)."""
    import torch
    n = int(params.n)
    fdt = torch.float64 if params.precision == LJ_PREC_FP64 else torch.float32
    _ck(load().lj_forces_static(ctypes.byref(params), _dev(x, torch.float64, (n, 3), "x"),
                                _dev(f, fdt, (n, 4), "f"), _stream_ptr(stream)), "lj_forces_static")


PEAK_FP32, PEAK_FP32X2, PEAK_FP64 = 0, 1, 2


def lj_measure_peak(kind: int) -> tuple[float, float, int]:
    """Measured FMA peak of the current device: (flop/s, ms of the timed
    launch, SM count); kind PEAK_FP32, PEAK_FP32X2 (packed pairs) or PEAK_FP64."""
    fl = ctypes.c_double()
    ms = ctypes.c_double()
    sms = ctypes.c_int32()
    _ck(load().lj_measure_peak(int(kind), ctypes.byref(fl), ctypes.byref(ms), ctypes.byref(sms)),
        "lj_measure_peak")
    return fl.value, ms.value, sms.value


def lj_check(ctx: Context) -> None:
    _ck(load().lj_check(ctx.handle), "lj_check")


def lj_set_timing(ctx: Context, enable: bool) -> None:
    _ck(load().lj_set_timing(ctx.handle, 1 if enable else 0), "lj_set_timing")


def lj_read_timing(ctx: Context) -> tuple[float, int, int]:
    """(force-kernel ms, timed force launches, kernels launched)."""
    ms = ctypes.c_double()
    nf = ctypes.c_int64()
    nk = ctypes.c_int64()
    _ck(load().lj_read_timing(ctx.handle, ctypes.byref(ms), ctypes.byref(nf), ctypes.byref(nk)),
        "lj_read_timing")
    return ms.value, nf.value, nk.value


# ---- checkpoint files ------------------------------------------------------
# One .npz per checkpoint: the parameters, x, v, f, whether f holds the forces
# of x, the step count, the in-cell order mode and, once the thermostat was
# seeded, its n rand48 stream states.  The cell arrays are not saved: they
# are a function of x and are rebuilt by the first step after loading.

CHECKPOINT_VERSION = 1
_PARAM_FIELDS = [name for name, _ in lj_params._fields_]
_RAND48_LIMIT = 1 << 48


def write_checkpoint(path, params: lj_params, x, v, f, *, steps: int = 0, forces_valid: bool = True,
                     deterministic: bool = False, rng=None) -> None:
    """Write a checkpoint file (host arrays: x, v (n, 3) float64, f (n, 4)
    float32 or float64 per the precision, rng (n,) uint64 or None)."""
    n = int(params.n)
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    fdt = np.float32 if params.precision == LJ_PREC_MIXED else np.float64
    f = np.asarray(f)
    if x.shape != (n, 3) or v.shape != (n, 3) or f.shape != (n, 4) or f.dtype != fdt:
        raise ValueError("checkpoint arrays do not match the parameters")
    arrays = {"version": np.int64(CHECKPOINT_VERSION),
              "params": np.array([getattr(params, k) for k in _PARAM_FIELDS], dtype=np.float64),
              "param_names": np.array(_PARAM_FIELDS),
              "x": x, "v": v, "f": f, "steps": np.int64(steps),
              "forces_valid": np.bool_(forces_valid), "deterministic": np.bool_(deterministic)}
    if rng is not None:
        rng = np.ascontiguousarray(rng).view(np.uint64) if np.asarray(rng).dtype == np.int64 else \
            np.ascontiguousarray(rng, dtype=np.uint64)
        if rng.shape != (n,) or np.any(rng >= _RAND48_LIMIT):
            raise ValueError("rng must hold n stream states below 2^48")
        arrays["rng"] = rng
    with open(path, "wb") as fh:
        np.savez(fh, **arrays)


def read_checkpoint(path) -> dict:
    """Read and validate a checkpoint file: a dict with params (lj_params),
    x, v, f, steps, forces_valid, deterministic and rng (None if absent)."""
    with np.load(path, allow_pickle=False) as z:
        if "version" not in z.files or int(z["version"]) != CHECKPOINT_VERSION:
            raise ValueError(f"{path}: not a version {CHECKPOINT_VERSION} checkpoint")
        names = [str(k) for k in z["param_names"]]
        if names != _PARAM_FIELDS:
            raise ValueError(f"{path}: parameter fields {names} differ from {_PARAM_FIELDS}")
        vals = dict(zip(names, z["params"].tolist()))
        params = lj_params(*[(int(vals[k]) if t is not ctypes.c_double else float(vals[k]))
                             for k, t in lj_params._fields_])
        out = {"params": params, "x": z["x"], "v": z["v"], "f": z["f"], "steps": int(z["steps"]),
               "forces_valid": bool(z["forces_valid"]), "deterministic": bool(z["deterministic"]),
               "rng": z["rng"] if "rng" in z.files else None}
    n = int(params.n)
    fdt = np.float32 if params.precision == LJ_PREC_MIXED else np.float64
    if (out["x"].shape != (n, 3) or out["v"].shape != (n, 3) or out["f"].shape != (n, 4)
            or out["x"].dtype != np.float64 or out["v"].dtype != np.float64 or out["f"].dtype != fdt):
        raise ValueError(f"{path}: arrays do not match the parameters")
    if out["rng"] is not None and (out["rng"].shape != (n,) or out["rng"].dtype != np.uint64
                                   or np.any(out["rng"] >= _RAND48_LIMIT)):
        raise ValueError(f"{path}: rng must hold n stream states below 2^48")
    return out


class System:
    """Convenience owner of a context and its device state (x, v, f).

    x, v are (n, 3) float64 CUDA tensors, f is (n, 4) float32 (mixed) or
    float64 (fp64)."""

    def __init__(self, x, v, box: float, *, eps=1.0, sigma=1.0, rc=2.5, dt=0.005, mass=1.0,
                 shift_mode=LJ_SHIFT_ENERGY, precision="mixed", flags=0, cell_subdiv=1, device=None, stream=None):
        import torch
        device = torch.device("cuda") if device is None else torch.device(device)
        self.x = torch.as_tensor(np.asarray(x, dtype=np.float64)).to(device).contiguous()
        n = self.x.shape[0]
        if v is None:
            self.v = torch.zeros((n, 3), dtype=torch.float64, device=device)
        else:
            self.v = torch.as_tensor(np.asarray(v, dtype=np.float64)).to(device).contiguous()
        self.params = make_params(n, box, eps, sigma, rc, dt, mass, shift_mode, precision, cell_subdiv, flags)
        self.ctx = Context(self.params, stream)
        self.f = torch.zeros((n, 4), dtype=self.ctx.force_dtype, device=device)
        self._forces_valid = False
        self.steps = 0
        self.deterministic = False
        self._rng_seeded = False

    @property
    def n(self) -> int:
        return self.ctx.n

    def forces(self, energy: bool = False):
        r = lj_forces(self.ctx, self.x, self.f, energy)
        self._forces_valid = True
        return r

    def step(self, nsteps: int) -> None:
        if not self._forces_valid:
            self.forces()
        lj_step(self.ctx, self.x, self.v, self.f, nsteps)
        self.steps += int(nsteps)

    def set_deterministic(self, enable: bool = True) -> None:
        lj_set_deterministic(self.ctx, enable)
        self.deterministic = bool(enable)

    def langevin_seed(self, seed: int) -> None:
        lj_langevin_seed(self.ctx, seed)
        self._rng_seeded = self.n > 0

    def langevin_step(self, nsteps: int, gamma: float, kT: float) -> None:
        if not self._forces_valid:
            self.forces()
        lj_langevin_step(self.ctx, self.x, self.v, self.f, nsteps, gamma, kT)
        self.steps += int(nsteps)

    def save(self, path) -> None:
        """Write a checkpoint of this system (synchronizes its stream)."""
        rng = lj_get_rng_state(self.ctx) if self._rng_seeded else None
        lj_check(self.ctx)
        rng = None if rng is None else rng.cpu().numpy().view(np.uint64)
        write_checkpoint(path, self.params, self.x.cpu().numpy(), self.v.cpu().numpy(), self.f.cpu().numpy(),
                         steps=self.steps, forces_valid=self._forces_valid, deterministic=self.deterministic,
                         rng=rng)

    @classmethod
    def load(cls, path, device=None, stream=None) -> "System":
        """A new system continuing from a checkpoint: same parameters, x, v,
        f, step count, in-cell order mode and thermostat series.  Tuning, the
        skin and graph replay are not part of a checkpoint; set them again."""
        import torch
        ck = read_checkpoint(path)
        p = ck["params"]
        s = cls(ck["x"], ck["v"], p.box, eps=p.eps, sigma=p.sigma, rc=p.rc, dt=p.dt, mass=p.mass,
                shift_mode=p.shift_mode, precision=p.precision, flags=p.flags, cell_subdiv=p.cell_subdiv,
                device=device, stream=stream)
        s.f.copy_(torch.from_numpy(ck["f"]))
        s._forces_valid = ck["forces_valid"]
        s.steps = ck["steps"]
        if ck["deterministic"]:
            s.set_deterministic(True)
        if ck["rng"] is not None and s.n > 0:
            lj_set_rng_state(s.ctx, torch.from_numpy(ck["rng"].view(np.int64)).to(s.x.device))
            s._rng_seeded = True
        lj_check(s.ctx)
        return s

    def energy(self):
        return lj_energy(self.ctx, self.x, self.v)

    def observables(self) -> dict:
        return lj_observables(self.ctx, self.x, self.v)

    def cells(self):
        import torch
        dev = self.x.device
        ncell = self.ctx.nc ** 3
        cell_of = torch.empty(self.n, dtype=torch.int32, device=dev)
        count = torch.empty(ncell, dtype=torch.int32, device=dev)
        start = torch.empty(ncell + 1, dtype=torch.int32, device=dev)
        perm = torch.empty(self.n, dtype=torch.int32, device=dev)
        lj_bin(self.ctx, self.x)
        lj_get_cells(self.ctx, cell_of, count, start, perm)
        return cell_of, count, start, perm

    def check(self) -> None:
        lj_check(self.ctx)

    def close(self) -> None:
        self.ctx.close()
