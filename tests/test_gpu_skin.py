"""Cell lists with a skin (Section 3.1): cells of side >= rc + skin rebuilt only
when some particle has moved half the skin.  The forces are those of the
exact cell list, so trajectories match the oracle's velocity Verlet (which
rebuilds every step) with the same tolerances as the plain step tests."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

from gpu_util import min_image

pytestmark = pytest.mark.gpu


def _liquid(seed, T=1.0, n_fcc=8):
    x, L = inputs.jittered_fcc(n_fcc, 0.8442, 0.08, seed)
    return x, inputs.velocities(x.shape[0], T, seed), L


@pytest.mark.parametrize("precision,skin,interval", [("fp64", 0.4, 0), ("mixed", 0.4, 0), ("fp64", 0.8, 0),
                                                     ("fp64", 0.3, 3), ("mixed", 0.6, 1)])
def test_skin_trajectory_matches_oracle(oracle_mod, precision, skin, interval):
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid(41, T=1.5)
    steps = 40 if precision == "fp64" else 20   # FP32 rounding grows along a chaotic trajectory
    xo, vo = x.copy(), v.copy()
    fo = oracle_mod.forces_cells(xo, L, mode=2)[0]
    oracle_mod.vv(xo, vo, fo, L, steps, mode=2)
    s = lj.System(x, v, L, precision=precision, shift_mode=2)
    lj.lj_set_skin(s.ctx, skin, interval)
    s.step(7)
    s.step(steps - 7)
    s.check()
    rebuilds, counted = lj.lj_skin_stats(s.ctx)
    xt, vt, ft = s.x.cpu().numpy(), s.v.cpu().numpy(), s.f.double().cpu().numpy()[:, :3]
    s.close()
    assert counted == steps
    if interval == 1:
        assert rebuilds == steps
    else:
        assert 1 <= rebuilds < steps
    xtol, vtol = (1e-10, 1e-9) if precision == "fp64" else (2e-6, 2e-4)
    assert np.abs(min_image(xt - xo, L)).max() <= xtol
    assert np.abs(vt - vo).max() <= vtol
    assert np.abs(ft - fo).max() <= (1e-8 if precision == "fp64" else 3e-4) * np.abs(fo).max()


def test_larger_skin_rebuilds_less():
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid(42, T=1.0, n_fcc=10)
    counts = []
    for skin in (0.2, 0.5, 1.0):
        s = lj.System(x, v, L)
        lj.lj_set_skin(s.ctx, skin)
        s.step(60)
        s.check()
        counts.append(lj.lj_skin_stats(s.ctx)[0])
        s.close()
    assert counts[0] > counts[1] > counts[2] >= 1


def test_skin_cells_and_back():
    """The grid follows the skin: n = int[L / (rc + skin)]; skin 0 restores
    the per-step rebuild with the original grid."""
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid(43)
    s = lj.System(x, v, L)
    n0 = s.ctx.nc
    lj.lj_set_skin(s.ctx, 0.5)
    assert s.ctx.nc == int(L // 3.0)
    cell_of, count, start, perm = (t.cpu().numpy() for t in s.cells())
    assert count.size == s.ctx.nc ** 3 and int(start[-1]) == x.shape[0]
    s.step(5)
    lj.lj_set_skin(s.ctx, 0.0)
    assert s.ctx.nc == n0
    s.step(5)
    s.check()
    s.close()


def test_skin_argument_errors():
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid(44)
    s = lj.System(x, v, L)
    for bad in (-0.1, float("nan")):
        with pytest.raises(lj.LJError) as ei:
            lj.lj_set_skin(s.ctx, bad)
        assert ei.value.code == lj.LJ_EINVAL
    with pytest.raises(lj.LJError) as ei:
        lj.lj_set_skin(s.ctx, L)              # fewer than 3 cells
    assert ei.value.code == lj.LJ_EBOX
    lj.lj_set_skin(s.ctx, 0.3)
    with pytest.raises(lj.LJError) as ei:
        lj.lj_set_tuning(s.ctx, 0)            # fused update bins every step
    assert ei.value.code == lj.LJ_EINVAL
    s.close()


def test_skin_with_subdivision_two(oracle_mod):
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid(45, T=1.2)
    xo, vo = x.copy(), v.copy()
    fo = oracle_mod.forces_cells(xo, L, mode=2)[0]
    oracle_mod.vv(xo, vo, fo, L, 20, mode=2)
    s = lj.System(x, v, L, precision="mixed", shift_mode=2, cell_subdiv=2)
    lj.lj_set_skin(s.ctx, 0.4)
    s.step(20)
    s.check()
    assert np.abs(min_image(s.x.cpu().numpy() - xo, L)).max() <= 2e-6
    s.close()
