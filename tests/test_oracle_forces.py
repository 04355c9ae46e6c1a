"""Pins of the oracle's forces: Eq. (n2_force) brute force, the Section 3
cell list, and physical invariants (Newton's third law, F = -grad E,
translation / permutation invariance, independence of the cell size)."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs


def _liquid(n_fcc, rho, seed, amp=0.08):
    return inputs.jittered_fcc(n_fcc, rho, amp, seed)


def test_two_body_closed_form(oracle_mod):
    # Two particles across the periodic boundary, separated by r along a
    # diagonal: f_0 = F(r) d/r, f_1 = -f_0 (Eq. n2_force).
    L = 9.0
    for mode in (0, 1, 2):
        for r in (0.97, 1.12, 1.6, 2.3):
            u = np.array([1.0, 2.0, -2.0]) / 3.0
            x = np.array([[0.2, 4.0, 8.9], [0.2, 4.0, 8.9]]) + 0.0
            x[1] = x[0] - r * u
            x[1] = np.mod(x[1], L)
            f, ep, E, W = oracle_mod.forces_brute(x, L, mode=mode)
            F, U = oracle_mod.pair(r, mode=mode)
            np.testing.assert_allclose(f[0], F * u, rtol=1e-12, atol=1e-13)
            np.testing.assert_allclose(f[1], -F * u, rtol=1e-12, atol=1e-13)
            assert E == pytest.approx(U, rel=1e-12, abs=1e-15)
            assert W == pytest.approx(r * F, rel=1e-12, abs=1e-15)
            np.testing.assert_allclose(ep, [U / 2, U / 2], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("n_fcc,rho,rc", [(2, 0.8442, 1.1), (5, 0.8442, 2.5), (8, 0.8442, 2.5),
                                          (6, 0.5, 2.5), (5, 1.0, 2.5)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_cells_equal_brute_force(oracle_mod, n_fcc, rho, rc, mode):
    x, L = _liquid(n_fcc, rho, 7 + n_fcc)
    fb, eb, Eb, Wb = oracle_mod.forces_brute(x, L, rc=rc, mode=mode)
    fc, ec, Ec, Wc = oracle_mod.forces_cells(x, L, rc=rc, mode=mode)
    scale = np.abs(fb).max()
    np.testing.assert_allclose(fc, fb, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(ec, eb, rtol=0, atol=1e-12 * np.abs(eb).max())
    assert Ec == pytest.approx(Eb, rel=1e-12)
    assert Wc == pytest.approx(Wb, rel=1e-12)


def test_cells_on_uniform_random_gas(oracle_mod):
    # Random (overlapping) gas at low density still matches brute force.
    L = 12.0
    x = inputs.uniform(300, L, 5)
    fb, _, Eb, _ = oracle_mod.forces_brute(x, L, mode=1)
    fc, _, Ec, _ = oracle_mod.forces_cells(x, L, mode=1)
    np.testing.assert_allclose(fc, fb, rtol=1e-12, atol=1e-12 * np.abs(fb).max())
    assert Ec == pytest.approx(Eb, rel=1e-12)


@pytest.mark.parametrize("k", [2, 3])
def test_independent_of_cell_subdivision(oracle_mod, k):
    x, L = _liquid(8, 0.8442, 11)
    f1, e1, E1, W1 = oracle_mod.forces_cells(x, L, mode=1, k=1)
    fk, ek, Ek, Wk = oracle_mod.forces_cells(x, L, mode=1, k=k)
    np.testing.assert_allclose(fk, f1, rtol=0, atol=1e-12 * np.abs(f1).max())
    assert Ek == pytest.approx(E1, rel=1e-12)


def test_newton_third_law(oracle_mod):
    x, L = _liquid(10, 0.8442, 3)
    f, _, _, _ = oracle_mod.forces_cells(x, L, mode=1)
    assert np.abs(f.sum(axis=0)).max() < 1e-10 * np.abs(f).max()


@pytest.mark.parametrize("mode", [1, 2])
def test_force_is_minus_energy_gradient(oracle_mod, mode):
    x, L = _liquid(5, 0.8442, 19)
    f, _, _, _ = oracle_mod.forces_cells(x, L, mode=mode)
    h = 1e-6
    rng = np.random.default_rng(0)
    for i in rng.choice(x.shape[0], 6, replace=False):
        for d in range(3):
            xp = x.copy(); xp[i, d] += h
            xm = x.copy(); xm[i, d] -= h
            Ep = oracle_mod.forces_cells(xp, L, mode=mode)[2]
            Em = oracle_mod.forces_cells(xm, L, mode=mode)[2]
            g = (Ep - Em) / (2 * h)
            assert f[i, d] == pytest.approx(-g, rel=1e-6, abs=1e-6)


def test_translation_and_axis_permutation(oracle_mod):
    x, L = _liquid(6, 0.8442, 23)
    f, ep, E, W = oracle_mod.forces_cells(x, L, mode=1)
    shift = np.array([3.3, -17.1, 0.77])
    f2, _, E2, _ = oracle_mod.forces_cells(x + shift, L, mode=1)
    np.testing.assert_allclose(f2, f, rtol=0, atol=1e-10 * np.abs(f).max())
    assert E2 == pytest.approx(E, rel=1e-12)
    f3, _, E3, _ = oracle_mod.forces_cells(x[:, [1, 2, 0]], L, mode=1)
    np.testing.assert_allclose(f3, f[:, [1, 2, 0]], rtol=0, atol=1e-10 * np.abs(f).max())
    perm = np.random.default_rng(1).permutation(x.shape[0])
    f4, _, _, _ = oracle_mod.forces_cells(x[perm], L, mode=1)
    np.testing.assert_allclose(f4, f[perm], rtol=0, atol=1e-10 * np.abs(f).max())


def test_energy_and_virial_bookkeeping(oracle_mod):
    x, L = _liquid(5, 0.8442, 29)
    f, ep, E, W = oracle_mod.forces_cells(x, L, mode=1)
    assert ep.sum() == pytest.approx(E, rel=1e-12)
    fi, ei = oracle_mod.force_one(x, L, 17, mode=1)
    np.testing.assert_allclose(fi, f[17], rtol=1e-12, atol=1e-12)
    assert ei == pytest.approx(ep[17], rel=1e-12)
    # FCC lattice: every site is equivalent, so every force vanishes by symmetry.
    xl, Ll = inputs.fcc(5, 0.8442)
    fl, epl, El, _ = oracle_mod.forces_cells(xl, Ll, mode=1)
    assert np.abs(fl).max() < 1e-11
    np.testing.assert_allclose(epl, epl[0], rtol=1e-12)


def test_box_too_small_rejected(oracle_mod):
    x = inputs.uniform(10, 7.0, 0)
    with pytest.raises(ValueError):
        oracle_mod.forces_cells(x, 7.0, rc=2.5)


def _dFdr(oracle_mod, r, mode, eps=1.0, sigma=1.0, h=1e-6):
    # dF/dr by central differences of the pinned pair force (not a retyped formula)
    Fp, _ = oracle_mod.pair(r + h, eps=eps, sigma=sigma, mode=mode)
    Fm, _ = oracle_mod.pair(r - h, eps=eps, sigma=sigma, mode=mode)
    return (Fp - Fm) / (2 * h)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (0.7, 1.1)])
def test_stiffness_two_and_three_body(oracle_mod, mode, eps, sigma):
    # K_i = sum_j |F'(r_ij)| + |F(r_ij)| / r_ij and S_i = sum_j |F(r_ij)| over
    # partners within rc, checked on hand-built configurations: the per-particle
    # bound of every mixed-precision parity test is built from them.
    L = 10.0
    u = np.array([2.0, -1.0, 2.0]) / 3.0
    w = np.array([0.0, 0.6, -0.8])
    r1, r2, r3 = 1.05, 1.9, 2.45
    # two bodies across the periodic boundary
    x = np.array([[9.7, 0.3, 5.0], [0.0, 0.0, 0.0]])
    x[1] = np.mod(x[0] + r1 * u, L)
    K, S = oracle_mod.stiffness(x, L, eps=eps, sigma=sigma, mode=mode)
    F1, _ = oracle_mod.pair(r1, eps=eps, sigma=sigma, mode=mode)
    k1 = abs(_dFdr(oracle_mod, r1, mode, eps, sigma)) + abs(F1) / r1
    np.testing.assert_allclose(K, [k1, k1], rtol=1e-7)
    np.testing.assert_allclose(S, [abs(F1), abs(F1)], rtol=1e-12)
    # three bodies: 0 has partners at r1 and r2; 1 and 2 are more than rc apart
    # (|r1 u - r2 w| > 2.5), so each has particle 0 only
    x3 = np.array([[5.0, 5.0, 5.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    x3[1] = x3[0] + r1 * u
    x3[2] = x3[0] + r2 * w
    assert np.linalg.norm(r1 * u - r2 * w) > 2.5
    K3, S3 = oracle_mod.stiffness(x3, L, eps=eps, sigma=sigma, mode=mode)
    F2, _ = oracle_mod.pair(r2, eps=eps, sigma=sigma, mode=mode)
    k2 = abs(_dFdr(oracle_mod, r2, mode, eps, sigma)) + abs(F2) / r2
    np.testing.assert_allclose(K3, [k1 + k2, k1, k2], rtol=1e-7)
    np.testing.assert_allclose(S3, [abs(F1) + abs(F2), abs(F1), abs(F2)], rtol=1e-12)
    # a partner at r3 < rc counts, one just beyond rc does not
    x4 = np.array([[5.0, 5.0, 5.0], [5.0 + r3, 5.0, 5.0], [5.0, 5.0 - 2.5 - 1e-9, 5.0]])
    K4, S4 = oracle_mod.stiffness(x4, L, eps=eps, sigma=sigma, mode=mode)
    F3, _ = oracle_mod.pair(r3, eps=eps, sigma=sigma, mode=mode)
    k3 = abs(_dFdr(oracle_mod, r3, mode, eps, sigma)) + abs(F3) / r3
    np.testing.assert_allclose(K4[:2], [k3, k3], rtol=1e-6)
    np.testing.assert_allclose(S4, [abs(F3), abs(F3), 0.0], rtol=1e-12, atol=0)
    assert K4[2] == 0.0
    # a subset of particles (idx) returns the same rows
    Ks, Ss = oracle_mod.stiffness(x3, L, eps=eps, sigma=sigma, mode=mode, idx=[2, 0])
    np.testing.assert_array_equal(Ks, K3[[2, 0]])
    np.testing.assert_array_equal(Ss, S3[[2, 0]])


@pytest.mark.parametrize("L", [7.0, 11.0])   # 2 cells per side: brute force; 4: the cell branch
def test_near_cutoff_band(oracle_mod, L):
    # A pair at |r - rc| < band flags both particles; pairs at 2 band from rc,
    # on either side, flag neither.  The band is on the distance r itself
    # (a band on r^2 would miss r = rc + 0.5 band for band << rc).
    rc, band = 2.5, 1e-3
    assert (oracle_mod.ncells(L, rc + band) >= 3) == (L > 8.0)
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    pairs = [(rc + 0.5 * band, True), (rc - 0.5 * band, True), (rc + 2 * band, False), (rc - 2 * band, False)]
    for r, flagged in pairs:
        x = np.array([[L - 0.2, 0.1, 0.5 * L], [0.0, 0.0, 0.0], [0.5 * L, 0.5 * L, 0.1]])
        x[1] = np.mod(x[0] + r * u, L)       # across the periodic boundary
        near = oracle_mod.near_cutoff(x, L, rc=rc, band=band)
        assert list(near) == [flagged, flagged, False], r
