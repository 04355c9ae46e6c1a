"""All-pairs GPU forces (Section 2, Eq. n2_force with the cutoff) against the
oracle's brute-force sum and against the GPU cell list.

Tolerance of the FP32-mixed all-pairs kernel: it takes absolute coordinates
relative to the box centre (|x| <= L/2, as the paper's N^2 code), so each
coordinate carries rounding up to 2^-25 L, the minimum-image shift another
2^-25 L and the difference 2^-24 rc: a pair vector is off by at most
dr = 3 * 2^-25 L + 2^-24 rc.  Per particle and component the force error is
then bounded by 1.5 dr K_i + 1e-5 S_i (K_i, S_i as in test_gpu_forces: the
stiffness and absolute-force sums; the factor 1.5 covers the three
components of the pair vector, the 1e-5 S_i term the FP32 sum and the
approximate reciprocal).  FP64: 1e-10 (|f| + f_rms)."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

from gpu_util import rel_rms

pytestmark = pytest.mark.gpu


def _n2(x, L, precision="mixed", mode=1, energy=True, **kw):
    from paper_0709_3225_gb300 import lj
    s = lj.System(x, None, L, precision=precision, shift_mode=mode, **kw)
    r = lj.lj_forces_n2(s.ctx, s.x, s.f, energy=energy)
    s.check()
    f = s.f.double().cpu().numpy()
    s.close()
    return f, r


def _check(x, L, oracle_mod, precision, mode=1, eps=1.0, sigma=1.0, rc=2.5):
    f, (e, w) = _n2(x, L, precision, mode, eps=eps, sigma=sigma, rc=rc)
    fo, epo, eo, wo = oracle_mod.forces_brute(x, L, eps=eps, sigma=sigma, rc=rc, mode=mode)
    near = oracle_mod.near_cutoff(x, L, rc=rc, band=1e-5 if precision == "mixed" else 1e-12)
    d = np.abs(f[:, :3] - fo).max(axis=1)
    K, S = oracle_mod.stiffness(x, L, eps=eps, sigma=sigma, rc=rc, mode=mode)
    if precision == "mixed":
        dr = 3 * 2.0 ** -25 * L + 2.0 ** -24 * rc
        bound = 1.5 * dr * K + 1e-5 * S
        assert rel_rms(f[:, :3], fo) <= max(1e-5, 2 * dr)
        etol = 2e-6
    else:
        frms = np.sqrt((fo ** 2).sum(axis=1).mean()) if fo.size else 0.0
        bound = 1e-10 * (np.abs(fo).max(axis=1) + frms)
        etol = 1e-11
    assert np.all(d[~near] <= bound[~near]), (d[~near] / np.maximum(bound[~near], 1e-300)).max()
    assert abs(e - eo) <= etol * max(np.abs(epo).sum(), 1e-300) + 1e-12
    assert abs(w - wo) <= etol * 0.5 * rc * S.sum() + 1e-12
    escale = np.abs(epo).max() if epo.size else 1.0
    assert np.all(np.abs(f[~near, 3] - epo[~near]) <= (1e-4 if precision == "mixed" else 1e-10) * escale)
    return f, fo


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_liquid_2k(oracle_mod, precision, mode):
    """2,048 particles: exactly four j tiles; several j-splits."""
    x, L = inputs.jittered_fcc(8, 0.8442, 0.1, 51)
    _check(x, L, oracle_mod, precision, mode)


@pytest.mark.parametrize("n", [2, 3, 300, 511, 513, 2500])
def test_ragged_sizes(oracle_mod, n):
    """Sizes below, at and across the tile and block boundaries."""
    x, L = inputs.lattice_gas(n, min(0.6, n / 8.0 ** 3), 60 + n)   # L >= 8 > 3 rc
    _check(x, L, oracle_mod, "mixed")
    _check(x, L, oracle_mod, "fp64")


def test_pair_across_the_boundary(oracle_mod):
    """Two particles that interact only through the periodic image."""
    L = 8.0
    x = np.array([[0.2, 4.0, 4.0], [7.1, 4.0, 4.0]])
    f, _ = _check(x, L, oracle_mod, "fp64")
    assert f[0, 0] > 0 and abs(f[0, 0] + f[1, 0]) < 1e-12


@pytest.mark.parametrize("eps,sigma,rc", [(0.9, 1.05, 2.5), (1.3, 0.9, 3.0)])
def test_other_parameters(oracle_mod, eps, sigma, rc):
    x, L = inputs.jittered_fcc(6, 0.8442, 0.08, 70)
    for mode in (1, 2):
        _check(x, L, oracle_mod, "mixed", mode, eps, sigma, rc)
        _check(x, L, oracle_mod, "fp64", mode, eps, sigma, rc)


def test_matches_the_cell_list():
    """All-pairs and cell-list forces agree (FP64: to rounding; FP32: within
    the all-pairs kernel's coordinate rounding)."""
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(10, 0.8442, 0.12, 71)
    for precision, tol in (("fp64", 1e-11), ("mixed", 2e-5)):
        s = lj.System(x, None, L, precision=precision)
        s.forces()
        fc = s.f.double().cpu().numpy()[:, :3]
        lj.lj_forces_n2(s.ctx, s.x, s.f)
        s.check()
        fn = s.f.double().cpu().numpy()[:, :3]
        s.close()
        assert rel_rms(fn, fc) <= tol


def test_empty_and_nonfinite():
    from paper_0709_3225_gb300 import lj
    f, (e, w) = _n2(np.zeros((0, 3)), 9.0)
    assert f.shape == (0, 4) and e == 0.0 and w == 0.0
    x, L = inputs.jittered_fcc(5, 0.8442, 0.05, 72)
    x[3, 2] = np.nan
    s = lj.System(x, None, L)
    lj.lj_forces_n2(s.ctx, s.x, s.f)
    with pytest.raises(lj.LJError) as ei:
        s.check()
    assert ei.value.code == lj.LJ_ENONFINITE
    s.close()


def test_repeated_calls_reuse_scratch(oracle_mod):
    """Later calls reuse the scratch of the first; results stay exact."""
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(5, 0.8442, 0.1, 73)
    s = lj.System(x, None, L, precision="fp64")
    for _ in range(3):
        lj.lj_forces_n2(s.ctx, s.x, s.f)
    s.check()
    fo = oracle_mod.forces_brute(x, L, mode=1)[0]
    assert np.abs(s.f.cpu().numpy()[:, :3] - fo).max() <= 1e-10 * (np.abs(fo).max() + 1)
    s.close()
