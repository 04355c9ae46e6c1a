"""Checkpoint / resume on the GPU: a system saved between two calls and
loaded into a new context continues exactly as the saved one does.  With the
deterministic in-cell order the forces do not depend on the binning atomics,
so the continuation is compared bit for bit (x, v, f), for velocity Verlet in
both precisions and for the Langevin thermostat, whose rand48 stream states
are part of the checkpoint."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

pytestmark = pytest.mark.gpu


def _liquid(n_fcc=8, seed=31):
    x, L = inputs.jittered_fcc(n_fcc, 0.8442, 0.1, seed)
    v = inputs.velocities(x.shape[0], 0.728, seed)
    return x, v, L


def _same(a, b):
    for name in ("x", "v", "f"):
        ta, tb = getattr(a, name).cpu().numpy(), getattr(b, name).cpu().numpy()
        assert np.array_equal(ta, tb), name


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_resume_continues_bitwise(tmp_path, precision):
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid()
    a = lj.System(x, v, L, precision=precision)
    a.set_deterministic(True)
    a.step(10)
    b = lj.System(x, v, L, precision=precision)
    b.set_deterministic(True)
    b.step(10)
    path = tmp_path / "vv.npz"
    b.save(path)
    b.close()
    a.step(10)
    c = lj.System.load(path)
    assert c.steps == 10 and c.deterministic
    c.step(10)
    a.check()
    c.check()
    assert c.steps == a.steps == 20
    _same(a, c)
    a.close()
    c.close()


def test_langevin_resume_continues_bitwise(tmp_path, oracle_mod):
    import torch
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid(seed=32)
    a = lj.System(x, v, L)
    a.set_deterministic(True)
    a.langevin_seed(2024)
    # the seeded state is the rand48 series after srand48(2024)
    st = lj.lj_get_rng_state(a.ctx)
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy().view(np.uint64),
                          oracle_mod.rand48_series(oracle_mod.srand48_state(2024), a.n))
    a.langevin_step(6, 1.0, 0.9)
    path = tmp_path / "langevin.npz"
    a.save(path)
    a.langevin_step(6, 1.0, 0.9)
    c = lj.System.load(path)
    c.langevin_step(6, 1.0, 0.9)
    a.check()
    c.check()
    _same(a, c)
    # the two contexts' series advanced alike
    sa, sc = lj.lj_get_rng_state(a.ctx), lj.lj_get_rng_state(c.ctx)
    torch.cuda.synchronize()
    assert torch.equal(sa, sc)
    a.close()
    c.close()


def test_rng_state_errors():
    import torch
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid()
    s = lj.System(x, v, L)
    with pytest.raises(lj.LJError) as ei:
        lj.lj_get_rng_state(s.ctx)             # not seeded yet
    assert ei.value.code == lj.LJ_EINVAL
    host = torch.zeros(s.n, dtype=torch.int64)
    with pytest.raises(TypeError):
        lj.lj_set_rng_state(s.ctx, host)         # the binding wants a device tensor
    # set, then get returns the same states
    st = torch.arange(1, s.n + 1, dtype=torch.int64, device="cuda") * 7919
    lj.lj_set_rng_state(s.ctx, st)
    got = lj.lj_get_rng_state(s.ctx)
    torch.cuda.synchronize()
    assert torch.equal(got, st)
    s.close()
