"""Pins of the oracle's rand48 generator (Section 4) and Langevin step.

rand48_series is pinned to the C library's srand48 / lrand48 / drand48
(an implementation outside this repository); rand48_jump to the serial
series; the Langevin step to velocity Verlet (gamma = 0), to exact damping
(kT = 0, free particles) and to equipartition (an ideal gas thermalises to
kT)."""
import ctypes
import ctypes.util

import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs


def _libc():
    name = ctypes.util.find_library("c")
    if name is None:
        pytest.skip("no C library to compare with")
    libc = ctypes.CDLL(name)
    if not hasattr(libc, "lrand48"):
        pytest.skip("C library without rand48")
    libc.srand48.argtypes = [ctypes.c_long]
    libc.srand48.restype = None
    libc.lrand48.restype = ctypes.c_long
    libc.drand48.restype = ctypes.c_double
    return libc


@pytest.mark.parametrize("seed", [0, 1, 12345, 2 ** 31 - 1, 987654321])
def test_series_matches_the_c_library(oracle_mod, seed):
    libc = _libc()
    n = 5000
    s = oracle_mod.rand48_series(oracle_mod.srand48_state(seed), 2 * n)
    libc.srand48(seed)
    lr = np.array([libc.lrand48() for _ in range(n)], np.int64)
    dr = np.array([libc.drand48() for _ in range(n)])
    assert np.array_equal(lr, (s[:n] >> np.uint64(17)).astype(np.int64))
    assert np.array_equal(dr, s[n:].astype(np.float64) * 2.0 ** -48)
    assert np.all(lr >= 0) and np.all(lr < 2 ** 31)


def test_series_state_is_48_bit(oracle_mod):
    s = oracle_mod.rand48_series(oracle_mod.srand48_state(77), 10000)
    assert int(s.max()) < 2 ** 48
    # the low bit of an LCG with odd c alternates
    assert np.all((s[1:] & np.uint64(1)) != (s[:-1] & np.uint64(1)))


@pytest.mark.parametrize("m", [1, 2, 3, 7, 64, 1000, 6144])
def test_jump_equals_the_serial_series(oracle_mod, m):
    A, C = oracle_mod.rand48_jump(m)
    x0 = oracle_mod.srand48_state(4242)
    s = oracle_mod.rand48_series(x0, m + 50)
    chain = np.concatenate([[np.uint64(x0)], s])
    for n in range(0, 50, 7):
        assert (A * int(chain[n]) + C) % 2 ** 48 == int(chain[n + m])


def test_jump_zero_is_identity(oracle_mod):
    assert oracle_mod.rand48_jump(0) == (1, 0)


def _free(n, L, seed):
    x = inputs.uniform(n, L, seed)
    return x, np.zeros_like(x), np.zeros_like(x)


def test_langevin_without_friction_is_velocity_verlet(oracle_mod):
    x, L = inputs.jittered_fcc(6, 0.8442, 0.08, 3)
    v = inputs.velocities(x.shape[0], 1.0, 3)
    f = oracle_mod.forces_cells(x, L, mode=2)[0]
    xa, va, fa = x.copy(), v.copy(), f.copy()
    xb, vb, fb = x.copy(), v.copy(), f.copy()
    oracle_mod.vv(xa, va, fa, L, 20, mode=2)
    oracle_mod.langevin(xb, vb, fb, L, 20, seed=9, gamma=0.0, kT=1.0, mode=2)
    d = xa - xb
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-12
    assert np.abs(va - vb).max() < 1e-11


def test_langevin_zero_temperature_damps_exactly(oracle_mod):
    """Free particles at kT = 0: each step multiplies v by exp(-gamma dt)."""
    n, L = 500, 20.0
    x, _, f = _free(n, L, 4)
    v = inputs.velocities(n, 1.0, 4)
    v0 = v.copy()
    gamma, dt, steps = 3.0, 0.005, 40
    oracle_mod.langevin(x, v, f, L, steps, seed=1, gamma=gamma, kT=0.0, dt=dt, eps=0.0)
    np.testing.assert_allclose(v, v0 * np.exp(-gamma * dt * steps), rtol=1e-12, atol=0)


def test_langevin_ideal_gas_thermalises(oracle_mod):
    """Equipartition: an ideal gas under the thermostat reaches m <v^2> = 3 kT
    (statistical error of the time average ~0.5 % here; bound 3 %)."""
    n, L = 4000, 30.0
    x, v, f = _free(n, L, 5)
    kT, mass = 1.3, 2.0
    oracle_mod.langevin(x, v, f, L, 150, seed=11, gamma=8.0, kT=kT, eps=0.0, mass=mass)
    temps = []
    for _ in range(10):
        oracle_mod.langevin(x, v, f, L, 20, seed=100 + len(temps), gamma=8.0, kT=kT, eps=0.0, mass=mass)
        temps.append(mass * (v * v).sum() / (3 * n))
    assert abs(np.mean(temps) / kT - 1.0) < 0.03
    assert abs(v.mean()) < 0.05
