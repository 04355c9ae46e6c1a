"""GPU rand48 (Section 4) bit for bit against the oracle's serial series, and
the Langevin thermostat against the oracle's BAOAB step.

Langevin tolerances: FP64 contexts compute the Box-Muller normals in FP64
(the oracle's libm and CUDA's functions differ by about an ulp), so a
20-step liquid trajectory agrees to 1e-10 in x and 1e-9 in v, as plain
velocity Verlet does.  FP32-mixed forms the normals in FP32 (relative error
~1e-7 of a unit normal, times c2 sqrt(kT/m) per step) on top of the FP32
pair forces, so the bounds are those of the mixed velocity-Verlet test:
2e-6 in x, 2e-4 in v."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

from gpu_util import min_image

pytestmark = pytest.mark.gpu


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("S", [1, 7, 1000, 6144])
def test_seed_is_the_series(oracle_mod, S):
    import torch
    from paper_0709_3225_gb300 import lj
    x0 = oracle_mod.srand48_state(2024)
    assert lj.lj_srand48_state(2024) == x0
    st = torch.empty(S, dtype=torch.int64, device="cuda")
    lj.lj_rand48_seed(st, x0)
    assert np.array_equal(_u64(st), oracle_mod.rand48_series(x0, S))


@pytest.mark.parametrize("S,R", [(6144, 10), (1, 100), (333, 17), (65536, 4)])
def test_lrand_and_drand_continue_the_series(oracle_mod, S, R):
    import torch
    from paper_0709_3225_gb300 import lj
    x0 = oracle_mod.srand48_state(77 + S)
    ser = oracle_mod.rand48_series(x0, 3 * R * S)
    st = torch.empty(S, dtype=torch.int64, device="cuda")
    lj.lj_rand48_seed(st, x0)
    a = lj.lj_rand48_lrand(st, R).cpu().numpy()
    b = lj.lj_rand48_drand(st, R).cpu().numpy()
    c = lj.lj_rand48_lrand(st, R).cpu().numpy()
    torch.cuda.synchronize()
    assert np.array_equal(a, (ser[:R * S] >> np.uint64(17)).astype(np.int32))
    assert np.array_equal(b, ser[R * S:2 * R * S].astype(np.float64) * 2.0 ** -48)
    assert np.array_equal(c, (ser[2 * R * S:] >> np.uint64(17)).astype(np.int32))
    # the state now holds the next S elements
    nxt = oracle_mod.rand48_series(int(ser[-1]), S)
    assert np.array_equal(_u64(st), nxt)


@pytest.mark.parametrize("m", [0, 1, 2, 6144, 1000003])
def test_jump_constants(oracle_mod, m):
    from paper_0709_3225_gb300 import lj
    assert lj.lj_rand48_jump(m) == oracle_mod.rand48_jump(m)


def test_argument_errors():
    import torch
    from paper_0709_3225_gb300 import lj
    st = torch.zeros(8, dtype=torch.int64, device="cuda")
    lib = lj.load()
    import ctypes
    assert lib.lj_rand48_lrand(ctypes.c_void_p(st.data_ptr()), -1, 1, ctypes.c_void_p(st.data_ptr()), None) == 1
    host = np.zeros(8, np.int64)
    assert lib.lj_rand48_seed(ctypes.c_void_p(host.ctypes.data), 8, 1, None) == 1
    assert lib.lj_rand48_jump(-3, None, None) == 1


def _liquid(seed):
    x, L = inputs.jittered_fcc(8, 0.8442, 0.08, seed)
    return x, inputs.velocities(x.shape[0], 1.0, seed), L


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_langevin_matches_oracle(oracle_mod, precision):
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid(31)
    gamma, kT, seed, steps = 2.0, 0.9, 555, 20
    xo, vo = x.copy(), v.copy()
    fo = oracle_mod.forces_cells(xo, L, mode=2)[0]
    oracle_mod.langevin(xo, vo, fo, L, steps, seed=seed, gamma=gamma, kT=kT, mode=2)
    s = lj.System(x, v, L, precision=precision, shift_mode=2)
    s.forces()
    lj.lj_langevin_seed(s.ctx, seed)
    lj.lj_langevin_step(s.ctx, s.x, s.v, s.f, 5, gamma, kT)
    lj.lj_langevin_step(s.ctx, s.x, s.v, s.f, steps - 5, gamma, kT)
    s.check()
    xt, vt = s.x.cpu().numpy(), s.v.cpu().numpy()
    s.close()
    xtol, vtol = (1e-10, 1e-9) if precision == "fp64" else (2e-6, 2e-4)
    assert np.abs(min_image(xt - xo, L)).max() <= xtol
    assert np.abs(vt - vo).max() <= vtol


def test_langevin_without_friction_is_lj_step():
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid(32)
    a = lj.System(x, v, L, precision="fp64", shift_mode=2)
    b = lj.System(x, v, L, precision="fp64", shift_mode=2)
    a.step(15)
    b.forces()
    lj.lj_langevin_seed(b.ctx, 1)
    lj.lj_langevin_step(b.ctx, b.x, b.v, b.f, 15, 0.0, 1.0)
    a.check()
    b.check()
    assert np.abs(min_image(a.x.cpu().numpy() - b.x.cpu().numpy(), L)).max() < 1e-11
    assert np.abs(a.v.cpu().numpy() - b.v.cpu().numpy()).max() < 1e-10
    a.close()
    b.close()


def test_langevin_thermalises_a_liquid():
    """The thermostat holds a cold-started liquid at kT: mean kinetic
    temperature over the last steps within 3 % (N = 32,000)."""
    import torch
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(20, 0.8442, 0.05, 33)
    s = lj.System(x, None, L)
    s.forces()
    lj.lj_langevin_seed(s.ctx, 99)
    kT = 1.4
    lj.lj_langevin_step(s.ctx, s.x, s.v, s.f, 400, 5.0, kT)
    temps = []
    for _ in range(10):
        lj.lj_langevin_step(s.ctx, s.x, s.v, s.f, 20, 5.0, kT)
        temps.append(float((s.v * s.v).sum()) / (3 * s.n))
    s.check()
    s.close()
    assert abs(np.mean(temps) / kT - 1.0) < 0.03


def test_langevin_needs_a_seed():
    from paper_0709_3225_gb300 import lj
    x, v, L = _liquid(34)
    s = lj.System(x, v, L)
    s.forces()
    with pytest.raises(lj.LJError) as ei:
        lj.lj_langevin_step(s.ctx, s.x, s.v, s.f, 1, 1.0, 1.0)
    assert ei.value.code == lj.LJ_EINVAL
    s.close()
