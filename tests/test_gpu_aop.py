"""The paper's fixed-capacity cell arrays (Section 3.1, lj_set_tuning kernel
4): same forces as the oracle (the FP32-mixed tolerances of
test_gpu_forces), virtual placeholders contribute nothing, and a cell over
the capacity of 32 is reported as LJ_EOVERFLOW."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

from gpu_util import dense_cluster_state, min_image, rel_rms

pytestmark = pytest.mark.gpu


def _aop_forces(x, L, mode=1, **kw):
    from paper_0709_3225_gb300 import lj
    s = lj.System(x, None, L, shift_mode=mode, **kw)
    lj.lj_set_tuning(s.ctx, 4)
    e, w = s.forces(energy=True)
    s.check()
    f = s.f.double().cpu().numpy()
    s.close()
    return f, e, w


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n_fcc,rho", [(8, 0.8442), (6, 0.3), (9, 1.0)])
def test_aop_matches_oracle(oracle_mod, mode, n_fcc, rho):
    x, L = inputs.jittered_fcc(n_fcc, rho, 0.08, 80 + n_fcc)
    f, e, w = _aop_forces(x, L, mode)
    fo, epo, eo, wo = oracle_mod.forces_cells(x, L, mode=mode)
    near = oracle_mod.near_cutoff(x, L, band=1e-5)
    K, S = oracle_mod.stiffness(x, L, mode=mode)
    d = np.abs(f[:, :3] - fo).max(axis=1)
    assert rel_rms(f[:, :3], fo) <= 1e-5
    assert np.all(d[~near] <= (6e-7 * K + 1e-5 * S)[~near])
    assert abs(e - eo) <= 2e-6 * np.abs(epo).sum() + 1e-12
    assert abs(w - wo) <= 2e-6 * 1.25 * S.sum() + 1e-12


def test_aop_trajectory(oracle_mod):
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(8, 0.8442, 0.08, 90)
    v = inputs.velocities(x.shape[0], 1.0, 90)
    xo, vo = x.copy(), v.copy()
    fo = oracle_mod.forces_cells(xo, L, mode=2)[0]
    oracle_mod.vv(xo, vo, fo, L, 15, mode=2)
    s = lj.System(x, v, L, shift_mode=2)
    lj.lj_set_tuning(s.ctx, 4)
    s.step(15)
    s.check()
    assert np.abs(min_image(s.x.cpu().numpy() - xo, L)).max() <= 2e-6
    assert np.abs(s.v.cpu().numpy() - vo).max() <= 2e-4
    s.close()


def test_aop_overflow_is_reported():
    from paper_0709_3225_gb300 import lj
    x, L = dense_cluster_state()
    s = lj.System(x, None, L)
    lj.lj_set_tuning(s.ctx, 4)
    lj.lj_forces(s.ctx, s.x, s.f)
    with pytest.raises(lj.LJError) as ei:
        s.check()
    assert ei.value.code == lj.LJ_EOVERFLOW
    s.close()


def test_aop_needs_mixed_and_27_cells():
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(8, 0.8442, 0.08, 91)
    for kw in ({"precision": "fp64"}, {"cell_subdiv": 2}):
        s = lj.System(x, None, L, **kw)
        with pytest.raises(lj.LJError) as ei:
            lj.lj_set_tuning(s.ctx, 4)
        assert ei.value.code == lj.LJ_EINVAL
        s.close()
