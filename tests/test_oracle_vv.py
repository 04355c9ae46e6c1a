"""Pins of the oracle's velocity-Verlet integration (Section 2, last
paragraph): time reversibility, momentum conservation and the second-order
scaling of its energy error with the time step."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs


def _state(n_fcc=5, rho=0.8442, T=0.728, seed=4):
    x, L = inputs.jittered_fcc(n_fcc, rho, 0.05, seed)
    v = inputs.velocities(x.shape[0], T, seed)
    return x, v, L


def test_time_reversibility(oracle_mod):
    x0, v0, L = _state()
    for mode in (1, 2):
        x, v = x0.copy(), v0.copy()
        f = oracle_mod.forces_cells(x, L, mode=mode)[0]
        oracle_mod.vv(x, v, f, L, 40, mode=mode)
        v *= -1.0
        oracle_mod.vv(x, v, f, L, 40, mode=mode)
        d = x - x0
        d -= L * np.round(d / L)
        assert np.abs(d).max() < 1e-8
        np.testing.assert_allclose(-v, v0, rtol=0, atol=1e-8)


def test_momentum_conserved_and_wrapped(oracle_mod):
    x, v, L = _state(seed=9)
    p0 = v.sum(axis=0)
    f = oracle_mod.forces_cells(x, L, mode=1)[0]
    oracle_mod.vv(x, v, f, L, 30, mode=1)
    assert np.abs(v.sum(axis=0) - p0).max() < 1e-11
    assert np.all(x >= 0.0) and np.all(x < L)


def test_energy_error_is_second_order(oracle_mod):
    """The energy fluctuation of velocity Verlet scales as dt^2: halving the
    step cuts it by ~4.  Uses the force-shifted potential (smooth at rc)."""
    x0, v0, L = _state(seed=13)
    spans = []
    for dt, nsteps in ((0.004, 50), (0.002, 100)):
        x, v = x0.copy(), v0.copy()
        f, _, E, _ = oracle_mod.forces_cells(x, L, mode=2)
        etot = [E + oracle_mod.ekin(v)]
        for _ in range(10):
            E, _ = oracle_mod.vv(x, v, f, L, nsteps // 10, dt=dt, mode=2)
            etot.append(E + oracle_mod.ekin(v))
        spans.append(np.max(np.abs(np.array(etot) - etot[0])))
    ratio = spans[0] / spans[1]
    assert 2.5 < ratio < 6.0, ratio


def test_single_step_matches_hand_update(oracle_mod):
    """One step equals v1/2 = v + dt/2 f, x1 = x + dt v1/2, v1 = v1/2 + dt/2 f(x1)."""
    x0, v0, L = _state(n_fcc=5, seed=21)
    dt = 0.005
    f0 = oracle_mod.forces_cells(x0, L, mode=1)[0]
    vh = v0 + 0.5 * dt * f0
    x1 = np.mod(x0 + dt * vh, L)
    f1 = oracle_mod.forces_cells(x1, L, mode=1)[0]
    v1 = vh + 0.5 * dt * f1
    x, v, f = x0.copy(), v0.copy(), f0.copy()
    oracle_mod.vv(x, v, f, L, 1, dt=dt, mode=1)
    np.testing.assert_allclose(x, x1, rtol=0, atol=1e-13)
    np.testing.assert_allclose(v, v1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(f, f1, rtol=0, atol=1e-10)


def test_input_state_pins():
    # FCC start: 4 n^3 sites, minimum separation a / sqrt(2) at rho = 0.8442.
    x, L = inputs.fcc(4, 0.8442)
    assert x.shape == (256, 3)
    a = L / 4
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1)) + np.eye(256) * 1e9
    assert r.min() == pytest.approx(a / np.sqrt(2), rel=1e-12)
    assert r.min() > 2 ** (1 / 6)
    v = inputs.velocities(256, 0.728, 1)
    assert np.abs(v.sum(axis=0)).max() < 1e-12
    assert (v ** 2).sum() / (3 * 256 - 3) == pytest.approx(0.728, rel=1e-12)


def test_relaxation_pins(oracle_mod):
    """Capped steepest descent: every move is at most dmax, the energy does
    not increase for a small step, and a force-free lattice stays put."""
    x0, L = inputs.lattice_gas(864, 0.85, 3, jitter=0.2)
    E0 = oracle_mod.forces_cells(x0, L, mode=1)[2]
    x1, _ = oracle_mod.relax(x0, L, 1, alpha=1e-3, dmax=0.05)
    d = x1 - x0
    d -= L * np.round(d / L)
    assert np.sqrt((d ** 2).sum(axis=1)).max() <= 0.05 + 1e-12
    energies = [E0]
    x = x0
    for _ in range(10):
        x, _ = oracle_mod.relax(x, L, 1, alpha=1e-3, dmax=0.05)
        energies.append(oracle_mod.forces_cells(x, L, mode=1)[2])
    assert np.all(np.diff(energies) <= 1e-9 * abs(E0))
    xl, Ll = inputs.fcc(5, 0.8442)
    xr, _ = oracle_mod.relax(xl, Ll, 5)
    np.testing.assert_allclose(xr, xl, rtol=0, atol=1e-11)


def test_lattice_gas_inputs():
    x, L = inputs.lattice_gas(5071, 0.726, 9)
    assert x.shape == (5071, 3)
    assert L == pytest.approx((5071 / 0.726) ** (1 / 3))
    e = inputs.ensemble(8, seed=1)
    assert len(e.n) == 8 and np.all((e.n >= 500) & (e.n <= 50000))
    assert np.all((e.rho >= 0.7) & (e.rho <= 0.9)) and np.all((e.temperature >= 0.7) & (e.temperature <= 1.5))


def test_all_pairs_and_cell_list_trajectories_agree(oracle_mod):
    # The fluid-2k workload (FCC 4*8^3, rho 0.8442, T 0.728), 100 steps of
    # velocity Verlet with the Section 2 all-pairs forces (k = 0) and with the
    # Section 3 cell list (k = 1): two independent force sums, one trajectory.
    x0, v0, L, w = inputs.workload_state("fluid-2k")
    traj = []
    for k in (0, 1):
        x, v = x0.copy(), v0.copy()
        f = oracle_mod.forces_brute(x, L)[0] if k == 0 else oracle_mod.forces_cells(x, L)[0]
        E, W = oracle_mod.vv(x, v, f, L, w.steps, dt=w.dt, k=k)
        traj.append((x, v, f, E, W))
    (xa, va, fa, Ea, Wa), (xb, vb, fb, Eb, Wb) = traj
    d = xa - xb
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-11
    assert np.abs(va - vb).max() < 1e-10
    assert np.abs(fa - fb).max() < 1e-9 * np.abs(fb).max()
    assert Ea == pytest.approx(Eb, rel=1e-12)
    assert Wa == pytest.approx(Wb, rel=1e-12)
