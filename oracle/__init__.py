"""FP64 CPU oracle for the Lennard-Jones cell-list MD path (test infrastructure).

This package is the slow, plain reference that the CUDA library is checked
against.  It is test infrastructure: only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code
with ``paper_0709_3225_gb300`` and never imports it.

The arithmetic lives in ``lj_oracle.c`` (plain C, IEEE double, built with
``-ffp-contract=off``); this module compiles it with gcc on first use and
wraps it with ctypes over numpy arrays.  Every function cites the passage of
van Meel et al., arXiv:0709.3225, that it follows.

Parity status of each function (what pins it, in tests/test_oracle_*.py):
  pair          -- special values at 2^(1/6) sigma, F = -dU/dr, asymptotes,
                   scaling laws (pinned)
  ncells        -- the paper's worked example L = 11, rc = 2.5 -> 4 (pinned)
  bin           -- independent interval test per particle, counts, edge
                   cases (pinned)
  forces_brute  -- Newton III, F = -grad E, two-body closed form (pinned)
  forces_cells  -- equals forces_brute; invariance under subdivision,
                   translation and axis permutation (pinned)
  vv            -- time reversibility, second-order energy error (pinned)
  rand48_series -- glibc's srand48 / lrand48 / drand48 sequences (pinned)
  rand48_jump   -- equals the serial series m steps ahead (pinned through
                   rand48_series)
  langevin      -- gamma = 0 is velocity Verlet; the ideal gas thermalises
                   to kT; Box-Muller normals have unit variance (pinned)
  stiffness     -- K and S of two- and three-body systems against the pair
                   force and its central-difference slope (pinned)
  near_cutoff   -- pairs at rc +- band/2 flagged, at rc +- 2 band not, in the
                   brute-force and the cell branch (pinned)
  observables   -- ideal gas P V = (2/3) E_kin; two-body virial r F(r); the
                   pressure equals -dE_pot/dV under uniform scaling; T of
                   hand-set velocities (pinned)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lj_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblj_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile lj_oracle.c into liblj_oracle.so (gcc, OpenMP if available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
            "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.or_pair.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, _D, _D]
        lib.or_pair.restype = None
        lib.or_ncells.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.or_ncells.restype = ctypes.c_int
        lib.or_bin.argtypes = [ctypes.c_int64, _D, ctypes.c_double, ctypes.c_int,
                               _I32, _I32, _I32, _I32]
        lib.or_bin.restype = None
        lib.or_forces_brute.argtypes = [ctypes.c_int64, _D] + [ctypes.c_double] * 4 + \
            [ctypes.c_int, _D, _D, _D, _D]
        lib.or_forces_brute.restype = None
        lib.or_forces_cells.argtypes = [ctypes.c_int64, _D] + [ctypes.c_double] * 4 + \
            [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        lib.or_forces_cells.restype = ctypes.c_int
        lib.or_force_one.argtypes = [ctypes.c_int64, _D] + [ctypes.c_double] * 4 + \
            [ctypes.c_int, ctypes.c_int64, _D, _D]
        lib.or_force_one.restype = None
        lib.or_near_cutoff.argtypes = [ctypes.c_int64, _D, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_double, _I32]
        lib.or_near_cutoff.restype = None
        lib.or_stiffness.argtypes = [ctypes.c_int64, _D] + [ctypes.c_double] * 4 + \
            [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, _D, _D]
        lib.or_stiffness.restype = None
        lib.or_pair_deriv.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, _D, _D, _D, _D]
        lib.or_pair_deriv.restype = None
        lib.or_forces_vjp.argtypes = [ctypes.c_int64, _D] + [ctypes.c_double] * 4 + \
            [ctypes.c_int, ctypes.c_int, _D, _D, _D]
        lib.or_forces_vjp.restype = ctypes.c_int
        lib.or_vv_adjoint.argtypes = [ctypes.c_int64, _D, _D] + [ctypes.c_double] * 4 + \
            [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _D, _D]
        lib.or_vv_adjoint.restype = ctypes.c_int
        lib.or_relax.argtypes = [ctypes.c_int64, _D, _D] + [ctypes.c_double] * 4 + \
            [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.or_relax.restype = ctypes.c_int
        lib.or_ekin.argtypes = [ctypes.c_int64, _D, ctypes.c_double]
        lib.or_ekin.restype = ctypes.c_double
        lib.or_vv.argtypes = [ctypes.c_int64, _D, _D, _D] + [ctypes.c_double] * 4 + \
            [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _D]
        lib.or_vv.restype = ctypes.c_int
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_set_threads.restype = ctypes.c_int
        _U64 = ctypes.POINTER(ctypes.c_uint64)
        lib.or_srand48_state.argtypes = [ctypes.c_int64]
        lib.or_srand48_state.restype = ctypes.c_uint64
        lib.or_rand48_series.argtypes = [ctypes.c_uint64, ctypes.c_int64, _U64]
        lib.or_rand48_series.restype = None
        lib.or_rand48_jump.argtypes = [ctypes.c_int64, _U64, _U64]
        lib.or_rand48_jump.restype = None
        lib.or_langevin.argtypes = [ctypes.c_int64, _D, _D, _D] + [ctypes.c_double] * 4 + \
            [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [ctypes.c_int, _U64, _D, _D]
        lib.or_langevin.restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_I32)


def _pos(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 2 or x.shape[1] != 3:
        raise ValueError("positions must have shape (n, 3)")
    return x


def set_threads(n: int = 0) -> int:
    """OpenMP threads for the cell-list loops (0 = leave as is); returns count."""
    return _load().or_set_threads(int(n))


def pair(r: float, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5,
         mode: int = 1) -> tuple[float, float]:
    """(F, U) of one pair at distance r (Section 2, LJ pair force and its
    truncated/shifted form; F = -dU/dr, positive repulsive)."""
    F = ctypes.c_double()
    U = ctypes.c_double()
    _load().or_pair(float(r), float(eps), float(sigma), float(rc), int(mode),
                    ctypes.byref(F), ctypes.byref(U))
    return F.value, U.value


def ncells(L: float, rc: float = 2.5, k: int = 1) -> int:
    """Cells per dimension n = int[k L / rc] (Section 3.2, worked example)."""
    return int(_load().or_ncells(float(L), float(rc), int(k)))


def bin_cells(x, L: float, nc: int):
    """Serial counting sort (Section 3.1 cell lists in CSR form).

    Returns (cell_of[n], count[nc^3], start[nc^3+1], perm[n]) as int32."""
    x = _pos(x)
    n = x.shape[0]
    ncell = nc ** 3
    cell_of = np.empty(n, np.int32)
    count = np.empty(ncell, np.int32)
    start = np.empty(ncell + 1, np.int32)
    perm = np.empty(n, np.int32)
    _load().or_bin(n, _dp(x), float(L), int(nc), _ip(cell_of), _ip(count), _ip(start), _ip(perm))
    return cell_of, count, start, perm


def forces_brute(x, L: float, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5,
                 mode: int = 1):
    """O(N^2) forces by Eq. (n2_force) at the minimum image.

    Returns (f[n,3], e_part[n], e_pot, virial)."""
    x = _pos(x)
    n = x.shape[0]
    f = np.empty((n, 3))
    ep = np.empty(n)
    E = ctypes.c_double()
    W = ctypes.c_double()
    _load().or_forces_brute(n, _dp(x), float(L), float(eps), float(sigma), float(rc), int(mode),
                            _dp(f), _dp(ep), ctypes.byref(E), ctypes.byref(W))
    return f, ep, E.value, W.value


def forces_cells(x, L: float, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5,
                 mode: int = 1, k: int = 1):
    """Cell-list forces (Section 3) over a (2k+1)^3 stencil.

    Returns (f[n,3], e_part[n], e_pot, virial)."""
    x = _pos(x)
    n = x.shape[0]
    f = np.empty((n, 3))
    ep = np.empty(n)
    E = ctypes.c_double()
    W = ctypes.c_double()
    rc_ = _load().or_forces_cells(n, _dp(x), float(L), float(eps), float(sigma), float(rc),
                                  int(mode), int(k), _dp(f), _dp(ep), ctypes.byref(E),
                                  ctypes.byref(W))
    if rc_ != 0:
        raise ValueError("box too small for the cell stencil (need nc >= 2k+1)")
    return f, ep, E.value, W.value


def force_one(x, L: float, i: int, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5,
              mode: int = 1):
    """Force and half pair energy on particle i alone, by definition (O(N))."""
    x = _pos(x)
    fi = np.empty(3)
    ei = ctypes.c_double()
    _load().or_force_one(x.shape[0], _dp(x), float(L), float(eps), float(sigma), float(rc),
                         int(mode), int(i), _dp(fi), ctypes.byref(ei))
    return fi, ei.value


def near_cutoff(x, L: float, rc: float = 2.5, band: float = 1e-5, k: int = 1) -> np.ndarray:
    """Boolean mask of particles with a partner at | r - rc | < band."""
    x = _pos(x)
    near = np.empty(x.shape[0], np.int32)
    _load().or_near_cutoff(x.shape[0], _dp(x), float(L), float(rc), int(k), float(band), _ip(near))
    return near.astype(bool)


def stiffness(x, L: float, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5, mode: int = 1,
              idx=None):
    """Per-particle (K, S): K = sum_j |F'(r_ij)| + |F(r_ij)|/r_ij and
    S = sum_j |F(r_ij)| over partners within rc (brute force) -- the
    sensitivity of f_i to rounding of the pair vectors and of the sum, for
    tolerance bounds only.  idx: optional particle subset."""
    x = _pos(x)
    n = x.shape[0]
    if idx is None:
        m, ip = n, None
    else:
        sel = np.ascontiguousarray(idx, dtype=np.int64)
        m, ip = sel.shape[0], sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    K = np.empty(m)
    S = np.empty(m)
    _load().or_stiffness(n, _dp(x), float(L), float(eps), float(sigma), float(rc), int(mode), ip, m,
                         _dp(K), _dp(S))
    return K, S


def pair_deriv(r: float, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5, mode: int = 1):
    """(F, dF/dr, dF/dsigma, dF/deps) of one pair (rc held fixed)."""
    out = [ctypes.c_double() for _ in range(4)]
    _load().or_pair_deriv(float(r), float(eps), float(sigma), float(rc), int(mode), *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def forces_vjp(x, L: float, g, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5, mode: int = 1,
               k: int = 1):
    """Vector-Jacobian product of the cell-list forces with g = dL/dF:
    returns (dL/dx (n, 3), dL/deps, dL/dsigma)."""
    x = _pos(x)
    g = _pos(g)
    dx = np.empty_like(x)
    dp = np.zeros(2)
    r = _load().or_forces_vjp(x.shape[0], _dp(x), float(L), float(eps), float(sigma), float(rc), int(mode),
                              int(k), _dp(g), _dp(dx), _dp(dp))
    if r != 0:
        raise ValueError("box too small for the cell stencil")
    return dx, float(dp[0]), float(dp[1])


def vv_adjoint(x0, v0, L: float, nsteps: int, gx, gv, dt: float = 0.005, eps: float = 1.0,
               sigma: float = 1.0, rc: float = 2.5, mode: int = 1, k: int = 1, mass: float = 1.0):
    """Adjoint of nsteps velocity-Verlet steps from (x0, v0): given dL/dx and
    dL/dv at the end, returns (dL/dx0, dL/dv0, dL/deps, dL/dsigma)."""
    x0 = _pos(x0)
    v0 = _pos(v0)
    ax = np.array(_pos(gx), copy=True)
    av = np.array(_pos(gv), copy=True)
    dp = np.zeros(2)
    r = _load().or_vv_adjoint(x0.shape[0], _dp(x0), _dp(v0), float(L), float(eps), float(sigma), float(rc),
                              int(mode), int(k), float(dt), float(mass), int(nsteps), _dp(ax), _dp(av), _dp(dp))
    if r != 0:
        raise ValueError("box too small for the cell stencil")
    return ax, av, float(dp[0]), float(dp[1])


def relax(x, L: float, nsteps: int, alpha: float = 1e-3, dmax: float = 0.05, eps: float = 1.0,
          sigma: float = 1.0, rc: float = 2.5, mode: int = 1, k: int = 1):
    """Capped steepest descent (x += alpha F per particle, move length capped
    at dmax, wrapped).  Returns (relaxed x, forces there)."""
    x = np.array(_pos(x), copy=True)
    f = np.empty_like(x)
    r = _load().or_relax(x.shape[0], _dp(x), _dp(f), float(L), float(eps), float(sigma), float(rc), int(mode),
                         int(k), int(nsteps), float(alpha), float(dmax))
    if r != 0:
        raise ValueError("box too small for the cell stencil")
    return x, f


def ekin(v, mass: float = 1.0) -> float:
    """Kinetic energy (1/2) m sum v^2."""
    v = _pos(v)
    return float(_load().or_ekin(v.shape[0], _dp(v), float(mass)))


def vv(x, v, f, L: float, nsteps: int, dt: float = 0.005, eps: float = 1.0,
       sigma: float = 1.0, rc: float = 2.5, mode: int = 1, k: int = 1, mass: float = 1.0):
    """Velocity Verlet (Section 2) for nsteps; x, v, f are updated IN PLACE
    (f must hold F(x) on entry).  k = 0 takes the forces from the all-pairs
    sum of Eq. (n2_force) (forces_brute) instead of the cell list.  Returns
    (e_pot, virial) at the end."""
    for a in (x, v, f):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                and a.ndim == 2 and a.shape[1] == 3):
            raise ValueError("x, v, f must be C-contiguous float64 arrays of shape (n, 3)")
    E = ctypes.c_double()
    W = ctypes.c_double()
    r = _load().or_vv(x.shape[0], _dp(x), _dp(v), _dp(f), float(L), float(eps), float(sigma),
                      float(rc), int(mode), int(k), float(dt), float(mass), int(nsteps),
                      ctypes.byref(E), ctypes.byref(W))
    if r != 0:
        raise ValueError("box too small for the cell stencil")
    return E.value, W.value


def srand48_state(seed: int) -> int:
    """x_0 of srand48(seed): (seed << 16) | 0x330E (low 32 bits of the seed)."""
    return int(_load().or_srand48_state(int(seed)))


def rand48_series(x0: int, n: int) -> np.ndarray:
    """x_1 .. x_n of the rand48 series (Section 4, Eq. lrand48) from x_0,
    serially, as uint64 (48-bit values).  lrand48 = x >> 17, drand48 = x 2^-48."""
    out = np.empty(int(n), np.uint64)
    _load().or_rand48_series(ctypes.c_uint64(int(x0)), int(n), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


def rand48_jump(m: int) -> tuple[int, int]:
    """(A, C) with x_{n+m} = (A x_n + C) mod 2^48 (Section 4, Eqs. lrand48m, AC)."""
    A = ctypes.c_uint64()
    C = ctypes.c_uint64()
    _load().or_rand48_jump(int(m), ctypes.byref(A), ctypes.byref(C))
    return int(A.value), int(C.value)


def langevin(x, v, f, L: float, nsteps: int, seed: int, gamma: float, kT: float, dt: float = 0.005,
             eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5, mode: int = 1, k: int = 1, mass: float = 1.0):
    """nsteps BAOAB Langevin steps (the stochastic thermostat of Section 1;
    scheme and random-number use documented in lj_oracle.c), normals from the
    rand48 series of srand48(seed).  x, v, f updated IN PLACE (f = F(x) on
    entry).  Returns (e_pot, virial) at the end."""
    for a in (x, v, f):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                and a.ndim == 2 and a.shape[1] == 3):
            raise ValueError("x, v, f must be C-contiguous float64 arrays of shape (n, 3)")
    n = x.shape[0]
    series = rand48_series(srand48_state(seed), 4 * n * int(nsteps))
    E = ctypes.c_double()
    W = ctypes.c_double()
    r = _load().or_langevin(n, _dp(x), _dp(v), _dp(f), float(L), float(eps), float(sigma), float(rc), int(mode),
                            int(k), float(dt), float(mass), float(gamma), float(kT), int(nsteps),
                            series.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(E),
                            ctypes.byref(W))
    if r != 0:
        raise ValueError("box too small for the cell stencil")
    return E.value, W.value


def observables(x, v, L: float, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5, mode: int = 1,
                k: int = 1, mass: float = 1.0) -> dict:
    """Thermodynamic observables of one state, by their definitions (FP64).

    The paper names energy conservation as the check on its single-precision
    runs (Section 5) and the temperature as what a thermostat holds (Section
    1); the quantities are the textbook ones (k_B = 1):
      E_kin = (1/2) m sum_i v_i^2,  E_pot = sum_{i<j} U(r_ij)  (Section 2),
      W     = sum_{i<j} r_ij F(r_ij)                        (the virial),
      T     = 2 E_kin / (3N - 3)   (momentum conserved: 3N - 3 degrees of
                                    freedom; 0 for N < 2),
      P     = (2 E_kin + W) / (3V),  V = L^3               (virial pressure).
    """
    x = _pos(x)
    n = x.shape[0]
    Ek = ekin(v, mass)
    if n > 0:
        _, _, Ep, W = forces_cells(x, L, eps, sigma, rc, mode, k)
    else:
        Ep, W = 0.0, 0.0
    T = 2.0 * Ek / (3 * n - 3) if n >= 2 else 0.0
    P = (2.0 * Ek + W) / (3.0 * L ** 3)
    return {"e_kin": Ek, "e_pot": Ep, "e_tot": Ek + Ep, "virial": W, "T": T, "P": P}
