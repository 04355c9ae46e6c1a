"""Pins of the oracle's observables (temperature, virial pressure): closed
forms and a thermodynamic identity that does not use the virial sum."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs


def test_ideal_gas(oracle_mod):
    # eps = 0: no interactions, W = 0, so P V = (2/3) E_kin = (N - 1) T.
    x, L = inputs.jittered_fcc(5, 0.8442, 0.1, 3)
    v = np.random.default_rng(4).normal(size=x.shape)
    o = oracle_mod.observables(x, v, L, eps=0.0)
    n = x.shape[0]
    assert o["virial"] == 0.0 and o["e_pot"] == 0.0
    assert o["e_kin"] == pytest.approx(0.5 * (v ** 2).sum(), rel=1e-14)
    assert o["P"] * L ** 3 == pytest.approx(2.0 * o["e_kin"] / 3.0, rel=1e-14)
    assert o["P"] * L ** 3 == pytest.approx((n - 1) * o["T"], rel=1e-14)


def test_temperature_of_hand_set_velocities(oracle_mod):
    # N = 4 particles with |v| = 0.5 each, mass 2: E_kin = 4 * (1/2) * 2 * 0.25 = 1,
    # T = 2 * 1 / (3 * 4 - 3) = 2/9.
    x = np.array([[1.0, 1.0, 1.0], [4.0, 1.0, 1.0], [1.0, 4.0, 1.0], [1.0, 1.0, 4.0]])
    v = np.array([[0.5, 0, 0], [-0.5, 0, 0], [0, 0.3, 0.4], [0, -0.3, -0.4]])
    o = oracle_mod.observables(x, v, 9.0, mass=2.0)
    assert o["e_kin"] == pytest.approx(1.0, rel=1e-15)
    assert o["T"] == pytest.approx(2.0 / 9.0, rel=1e-15)
    assert oracle_mod.observables(x[:1], v[:1], 9.0)["T"] == 0.0


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_two_body_pressure(oracle_mod, mode):
    # Two particles at rest a distance r apart: W = r F(r), P = r F(r) / (3 L^3).
    L, r = 8.0, 1.3
    x = np.array([[0.5, 7.9, 4.0], [0.0, 0.0, 0.0]])
    x[1] = np.mod(x[0] + r * np.array([0.6, 0.0, 0.8]), L)
    o = oracle_mod.observables(x, np.zeros_like(x), L, mode=mode)
    F, U = oracle_mod.pair(r, mode=mode)
    assert o["virial"] == pytest.approx(r * F, rel=1e-12)
    assert o["P"] == pytest.approx(r * F / (3 * L ** 3), rel=1e-12)
    assert o["e_pot"] == pytest.approx(U, rel=1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_pressure_is_minus_volume_derivative_of_energy(oracle_mod, mode):
    # At rest, P = -dE_pot/dV under a uniform scaling of positions and box
    # (x -> lam x, L -> lam L, V = lam^3 L^3): a check of the virial sum that
    # uses only the pinned potential energy.
    x, L = inputs.jittered_fcc(5, 0.8442, 0.1, 11)
    o = oracle_mod.observables(x, np.zeros_like(x), L, mode=mode)
    h = 1e-6
    Ep = oracle_mod.forces_cells(x * (1 + h), L * (1 + h), mode=mode)[2]
    Em = oracle_mod.forces_cells(x * (1 - h), L * (1 - h), mode=mode)[2]
    dV = (L * (1 + h)) ** 3 - (L * (1 - h)) ** 3
    assert o["P"] == pytest.approx(-(Ep - Em) / dV, rel=1e-6)
