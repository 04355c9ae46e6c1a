"""Pins of the oracle's pair interaction (Section 2, LJ pair force and its
truncated / shifted form) against facts that do not come from the oracle:
the position and depth of the LJ minimum, F = -dU/dr, the r^-12 and r^-6
asymptotes, the eps/sigma scaling laws and the strict cutoff."""
import math

import numpy as np
import pytest

RMIN = 2.0 ** (1.0 / 6.0)


@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (0.9, 1.05), (2.5, 0.8)])
def test_minimum_at_two_to_the_sixth(oracle_mod, eps, sigma):
    # The LJ well: zero force at r = 2^(1/6) sigma and energy -eps there.
    F0, U0 = oracle_mod.pair(RMIN * sigma, eps, sigma, rc=10.0, mode=0)
    assert abs(F0) < 1e-12 * eps / sigma
    assert U0 == pytest.approx(-eps, rel=1e-14)
    # Energy shift moves U but not F.
    F1, U1 = oracle_mod.pair(RMIN * sigma, eps, sigma, rc=2.5 * sigma, mode=1)
    assert abs(F1) < 1e-12 * eps / sigma
    _, Uc = oracle_mod.pair(2.5 * sigma * (1 - 1e-15), eps, sigma, rc=10.0, mode=0)
    assert U1 + Uc == pytest.approx(-eps, rel=1e-12)
    # Repulsive inside the minimum, attractive outside.
    assert oracle_mod.pair(0.95 * RMIN * sigma, eps, sigma, 10.0, 0)[0] > 0
    assert oracle_mod.pair(1.05 * RMIN * sigma, eps, sigma, 10.0, 0)[0] < 0


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (0.9, 1.05)])
def test_force_is_minus_energy_derivative(oracle_mod, mode, eps, sigma):
    rc = 2.5
    h = 1e-6
    for r in np.linspace(0.85, 2.45, 33):
        F, _ = oracle_mod.pair(r, eps, sigma, rc, mode)
        up = oracle_mod.pair(r + h, eps, sigma, rc, mode)[1]
        um = oracle_mod.pair(r - h, eps, sigma, rc, mode)[1]
        dudr = (up - um) / (2 * h)
        assert F == pytest.approx(-dudr, rel=1e-7, abs=1e-8)


def test_power_law_asymptotes(oracle_mod):
    # Short range: U * (r/sigma)^12 -> 4 eps; long range: U * (r/sigma)^6 -> -4 eps.
    eps, sigma = 1.7, 1.3
    r = 0.02 * sigma
    assert oracle_mod.pair(r, eps, sigma, 100.0, 0)[1] * (r / sigma) ** 12 == pytest.approx(4 * eps, rel=1e-9)
    r = 60.0 * sigma
    assert oracle_mod.pair(r, eps, sigma, 100.0, 0)[1] * (r / sigma) ** 6 == pytest.approx(-4 * eps, rel=1e-9)
    # Force asymptotes: F * (r/sigma)^13 -> 48 eps / sigma and F * (r/sigma)^7 -> -24 eps / sigma.
    r = 0.02 * sigma
    assert oracle_mod.pair(r, eps, sigma, 100.0, 0)[0] * (r / sigma) ** 13 == pytest.approx(48 * eps / sigma, rel=1e-9)
    r = 60.0 * sigma
    assert oracle_mod.pair(r, eps, sigma, 100.0, 0)[0] * (r / sigma) ** 7 == pytest.approx(-24 * eps / sigma, rel=1e-9)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_scaling_laws(oracle_mod, mode):
    # Dimensional analysis: U(r; eps, sigma, rc) = eps U(r/sigma; 1, 1, rc/sigma),
    # F(r; eps, sigma, rc) = (eps/sigma) F(r/sigma; 1, 1, rc/sigma).
    # This is what fixes the 1/sigma factor that the printed force lacks.
    eps, sigma, rc = 0.9, 1.05, 2.5
    for r in [0.9, 1.1, 1.5, 2.0, 2.4]:
        F, U = oracle_mod.pair(r, eps, sigma, rc, mode)
        F1, U1 = oracle_mod.pair(r / sigma, 1.0, 1.0, rc / sigma, mode)
        assert U == pytest.approx(eps * U1, rel=1e-13, abs=1e-15)
        assert F == pytest.approx(eps / sigma * F1, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_strict_cutoff(oracle_mod, mode):
    assert oracle_mod.pair(2.5, 1.0, 1.0, 2.5, mode) == (0.0, 0.0)
    assert oracle_mod.pair(3.0, 1.0, 1.0, 2.5, mode) == (0.0, 0.0)
    assert oracle_mod.pair(2.5 * (1 - 1e-15), 1.0, 1.0, 2.5, mode) != (0.0, 0.0)


def test_shift_modes(oracle_mod):
    rc = 2.5
    below = rc * (1 - 1e-12)
    F0c, U0c = oracle_mod.pair(below, 1.0, 1.0, rc, 0)
    # Energy shift: continuous energy at rc, constant offset from the plain form.
    assert abs(oracle_mod.pair(below, 1.0, 1.0, rc, 1)[1]) < 1e-12
    for r in [0.95, 1.3, 2.0]:
        F0, U0 = oracle_mod.pair(r, 1.0, 1.0, rc, 0)
        F1, U1 = oracle_mod.pair(r, 1.0, 1.0, rc, 1)
        assert F1 == F0
        assert U1 - U0 == pytest.approx(-U0c, rel=1e-10)
    # Force shift (the paper's form): force and energy both vanish at rc.
    F2c, U2c = oracle_mod.pair(below, 1.0, 1.0, rc, 2)
    assert abs(F2c) < 1e-10 and abs(U2c) < 1e-10
    for r in [0.95, 1.3, 2.0]:
        F0, _ = oracle_mod.pair(r, 1.0, 1.0, rc, 0)
        F2, _ = oracle_mod.pair(r, 1.0, 1.0, rc, 2)
        assert F2 - F0 == pytest.approx(-F0c, rel=1e-10)
    # The plain LJ force at rc is attractive and small (a few percent of eps/sigma).
    assert -0.1 < F0c < 0 and -0.1 < U0c < 0
