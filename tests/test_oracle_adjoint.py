"""Pins of the oracle's derivatives (force VJP / Hessian-vector product,
parameter gradients, adjoint velocity Verlet) against finite differences of
the oracle's own forward functions, which are pinned separately."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (0.9, 1.05)])
def test_pair_derivatives_by_finite_differences(oracle_mod, mode, eps, sigma):
    h = 1e-6
    for r in np.linspace(0.9, 2.4, 16):
        F, dFdr, dFds, dFde = oracle_mod.pair_deriv(r, eps, sigma, 2.5, mode)
        assert F == pytest.approx(oracle_mod.pair(r, eps, sigma, 2.5, mode)[0], rel=1e-12, abs=1e-14)
        fr = (oracle_mod.pair(r + h, eps, sigma, 2.5, mode)[0] - oracle_mod.pair(r - h, eps, sigma, 2.5, mode)[0]) / (2 * h)
        fs = (oracle_mod.pair(r, eps, sigma + h, 2.5, mode)[0] - oracle_mod.pair(r, eps, sigma - h, 2.5, mode)[0]) / (2 * h)
        fe = (oracle_mod.pair(r, eps + h, sigma, 2.5, mode)[0] - oracle_mod.pair(r, eps - h, sigma, 2.5, mode)[0]) / (2 * h)
        assert dFdr == pytest.approx(fr, rel=1e-6, abs=1e-7)
        assert dFds == pytest.approx(fs, rel=1e-6, abs=1e-7)
        assert dFde == pytest.approx(fe, rel=1e-6, abs=1e-7)


def _state(n_fcc=5, seed=3, amp=0.08):
    x, L = inputs.jittered_fcc(n_fcc, 0.8442, amp, seed)
    return x, L


def _smooth_state(oracle_mod, seed):
    """A jittered lattice with no pair within 2e-5 of rc (finite differences
    of +-1e-6 then never cross the cutoff); the first seed from `seed` on."""
    while True:
        x, L = _state(seed=seed)
        if not oracle_mod.near_cutoff(x, L, band=2e-5).any():
            return x, L
        seed += 1000


@pytest.mark.parametrize("mode", [1, 2])
def test_vjp_against_finite_differences(oracle_mod, mode):
    x, L = _smooth_state(oracle_mod, 3)
    rng = np.random.default_rng(1)
    g = rng.standard_normal(x.shape)
    eps, sigma = 0.9, 1.05
    dx, de, ds = oracle_mod.forces_vjp(x, L, g, eps=eps, sigma=sigma, mode=mode)

    def loss(xx, e=eps, s=sigma):
        return float((g * oracle_mod.forces_cells(xx, L, eps=e, sigma=s, mode=mode)[0]).sum())

    h = 1e-6
    for i in rng.choice(x.shape[0], 5, replace=False):
        for q in range(3):
            xp = x.copy(); xp[i, q] += h
            xm = x.copy(); xm[i, q] -= h
            assert dx[i, q] == pytest.approx((loss(xp) - loss(xm)) / (2 * h), rel=2e-6, abs=2e-6)
    assert de == pytest.approx((loss(x, e=eps + h) - loss(x, e=eps - h)) / (2 * h), rel=1e-6)
    assert ds == pytest.approx((loss(x, s=sigma + h) - loss(x, s=sigma - h)) / (2 * h), rel=1e-6)
    # the force Jacobian is symmetric: the VJP equals the directional derivative along g
    f_p = oracle_mod.forces_cells(x + h * g, L, eps=eps, sigma=sigma, mode=mode)[0]
    f_m = oracle_mod.forces_cells(x - h * g, L, eps=eps, sigma=sigma, mode=mode)[0]
    jg = (f_p - f_m) / (2 * h)
    np.testing.assert_allclose(dx, jg, rtol=0, atol=1e-5 * np.abs(dx).max())


def test_vjp_zero_for_zero_cotangent(oracle_mod):
    x, L = _state(seed=5)
    dx, de, ds = oracle_mod.forces_vjp(x, L, np.zeros_like(x))
    assert np.all(dx == 0) and de == 0 and ds == 0


def test_vv_adjoint_against_finite_differences(oracle_mod):
    """Loss = a . x(T) + b . v(T) after 15 force-shifted steps."""
    x0, L = _state(seed=7)
    v0 = inputs.velocities(x0.shape[0], 0.728, 7)
    rng = np.random.default_rng(2)
    a = rng.standard_normal(x0.shape)
    b = rng.standard_normal(x0.shape)
    nsteps, eps, sigma, mode = 15, 0.95, 1.02, 2

    def loss(xx, vv, e=eps, s=sigma):
        x, v = xx.copy(), vv.copy()
        f = oracle_mod.forces_cells(x, L, eps=e, sigma=s, mode=mode)[0]
        oracle_mod.vv(x, v, f, L, nsteps, eps=e, sigma=s, mode=mode)
        d = x - x0
        d -= L * np.round(d / L)            # unwrapped displacement
        return float((a * (x0 + d)).sum() + (b * v).sum())

    gx0, gv0, de, ds = oracle_mod.vv_adjoint(x0, v0, L, nsteps, a, b, eps=eps, sigma=sigma, mode=mode)
    h = 1e-6
    assert de == pytest.approx((loss(x0, v0, e=eps + h) - loss(x0, v0, e=eps - h)) / (2 * h), rel=2e-6)
    assert ds == pytest.approx((loss(x0, v0, s=sigma + h) - loss(x0, v0, s=sigma - h)) / (2 * h), rel=2e-6)
    for i in rng.choice(x0.shape[0], 3, replace=False):
        for q in range(3):
            xp = x0.copy(); xp[i, q] += h
            xm = x0.copy(); xm[i, q] -= h
            assert gx0[i, q] == pytest.approx((loss(xp, v0) - loss(xm, v0)) / (2 * h), rel=1e-5, abs=1e-5)
            vp = v0.copy(); vp[i, q] += h
            vm = v0.copy(); vm[i, q] -= h
            assert gv0[i, q] == pytest.approx((loss(x0, vp) - loss(x0, vm)) / (2 * h), rel=1e-5, abs=1e-5)
