"""Error paths through the C ABI on a GPU: latched device errors, argument
checks.  Nothing here faults or hangs the GPU: every bad pointer is rejected
on the host before a kernel sees it."""
import ctypes

import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_nonfinite_position_is_reported():
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(6, 0.8442, 0.05, 1)
    x[17, 1] = np.nan
    x[40, 0] = np.inf
    s = lj.System(x, None, L)
    lj.lj_forces(s.ctx, s.x, s.f)        # queued; the kernel latches the error
    with pytest.raises(lj.LJError) as ei:
        s.check()
    assert ei.value.code == lj.LJ_ENONFINITE
    s.check()                             # the latch is cleared by the check
    with pytest.raises(lj.LJError) as ei:
        s.forces(energy=True)             # synchronizing call reports it directly
    assert ei.value.code == lj.LJ_ENONFINITE
    s.close()


def test_box_too_small():
    from paper_0709_3225_gb300 import lj
    with pytest.raises(lj.LJError) as ei:
        lj.System(np.zeros((4, 3)), None, 7.0)
    assert ei.value.code == lj.LJ_EBOX


def test_binding_rejects_bad_tensors():
    import torch
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(6, 0.8442, 0.05, 1)
    s = lj.System(x, None, L)
    with pytest.raises(TypeError):
        lj.lj_bin(s.ctx, torch.zeros((s.n, 3), dtype=torch.float64))             # CPU tensor
    with pytest.raises(TypeError):
        lj.lj_bin(s.ctx, torch.zeros((s.n, 3), dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        lj.lj_bin(s.ctx, torch.zeros((s.n + 1, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        lj.lj_forces(s.ctx, s.x, torch.zeros((s.n, 8), dtype=torch.float32, device="cuda")[:, ::2])
    s.close()


def test_c_abi_rejects_host_and_misaligned_pointers():
    import torch
    from paper_0709_3225_gb300 import lj
    lib = lj.load()
    x, L = inputs.jittered_fcc(6, 0.8442, 0.05, 1)
    s = lj.System(x, None, L)
    host = np.zeros((s.n, 3))
    assert lib.lj_bin(s.ctx.handle, ctypes.c_void_p(host.ctypes.data)) == lj.LJ_EINVAL
    big = torch.zeros(3 * s.n + 8, dtype=torch.float64, device="cuda")
    assert lib.lj_bin(s.ctx.handle, ctypes.c_void_p(big.data_ptr() + 4)) == lj.LJ_EINVAL
    f = torch.zeros(4 * s.n + 8, dtype=torch.float32, device="cuda")
    assert lib.lj_forces(s.ctx.handle, ctypes.c_void_p(s.x.data_ptr()), ctypes.c_void_p(f.data_ptr() + 8),
                         None, None) == lj.LJ_EINVAL
    assert lib.lj_step(s.ctx.handle, ctypes.c_void_p(s.x.data_ptr()), ctypes.c_void_p(s.v.data_ptr()),
                       ctypes.c_void_p(s.f.data_ptr()), -1) == lj.LJ_EINVAL
    out = (ctypes.c_double * 3)()
    assert lib.lj_energy(s.ctx.handle, ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(s.v.data_ptr()),
                         out) == lj.LJ_EINVAL
    s.check()
    s.close()


def test_context_reuse_and_streams():
    """Two contexts on two streams give identical results to one context."""
    import torch
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(8, 0.8442, 0.08, 3)
    ref = lj.System(x, None, L, precision="fp64")
    ref.forces()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        other = lj.System(x, None, L, precision="fp64", stream=st)
        other.forces()
    st.synchronize()
    assert torch.allclose(ref.f, other.f, rtol=0, atol=1e-12)
    ref.close()
    other.close()


@pytest.mark.parametrize("kernel,grab", [(3, 0), (3, 4), (1, 0), (7, 4), (7, 0)])
def test_nonfinite_particles_go_to_the_extra_cell(oracle_mod, kernel, grab):
    """Non-finite particles are binned past the grid: the finite ones keep
    their exact cells and forces, and the error is still reported."""
    from paper_0709_3225_gb300 import lj
    from gpu_util import rel_rms
    x, L = inputs.jittered_fcc(8, 0.8442, 0.05, 3)
    bad = [5, 300, 1999]
    x[bad[0], 0] = np.nan
    x[bad[1], 2] = -np.inf
    x[bad[2], 1] = np.inf
    good = np.setdiff1d(np.arange(x.shape[0]), bad)
    s = lj.System(x, None, L)
    lj.lj_set_tuning(s.ctx, kernel, 0, grab)
    lj.lj_forces(s.ctx, s.x, s.f)
    with pytest.raises(lj.LJError) as ei:
        s.check()
    assert ei.value.code == lj.LJ_ENONFINITE
    cell_of, count, start, perm = (t.cpu().numpy() for t in s.cells())
    with pytest.raises(lj.LJError):
        s.check()
    ncell = s.ctx.nc ** 3
    assert np.all(cell_of[bad] == ncell)
    assert int(start[ncell]) == len(good) and int(count.sum()) == len(good)
    assert sorted(perm[len(good):].tolist()) == bad
    want = oracle_mod.bin_cells(np.ascontiguousarray(x[good]), L, s.ctx.nc)[0]
    assert np.array_equal(cell_of[good], want)
    fo = oracle_mod.forces_cells(np.ascontiguousarray(x[good]), L, mode=1)[0]
    fg = s.f.double().cpu().numpy()[good, :3]
    assert rel_rms(fg, fo) <= 1e-5
    s.close()


def test_nonfinite_particle_in_persistent_steps():
    """Steps through the persistent one-replica batch (tuning kernel 6)
    report a non-finite particle through lj_check like the regular path, and
    the context steps on normally once the state is finite again."""
    import torch
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(8, 0.8442, 0.05, 5)
    v = inputs.velocities(x.shape[0], 0.7, 5)
    s = lj.System(x, v, L)
    lj.lj_set_tuning(s.ctx, 6, 0, 1)
    s.forces()
    s.step(3)
    s.check()
    x_ok, v_ok, f_ok = s.x.clone(), s.v.clone(), s.f.clone()
    s.x[11, 2] = float("nan")
    s.step(2)
    with pytest.raises(lj.LJError) as ei:
        s.check()
    assert ei.value.code == lj.LJ_ENONFINITE
    s.x.copy_(x_ok)
    s.v.copy_(v_ok)
    s.f.copy_(f_ok)
    s.step(4)
    s.check()
    assert bool(torch.isfinite(s.x).all())
    s.close()


def test_nonfinite_replica_particle_is_isolated(oracle_mod):
    from paper_0709_3225_gb300 import lj
    from gpu_util import rel_rms
    e = inputs.ensemble(3, seed=9, n_lo=600, n_hi=1500)
    xs, vs = inputs.ensemble_state(e)
    xs[1] = xs[1].copy()
    xs[1][7, 0] = np.nan
    b = lj.Batch(xs, vs, e.box)
    b.forces()
    with pytest.raises(lj.LJError) as ei:
        b.check()
    assert ei.value.code == lj.LJ_ENONFINITE
    f = b.f.double().cpu().numpy()[:, :3]
    for r in (0, 2):
        fo = oracle_mod.forces_cells(xs[r], e.box[r], mode=1)[0]
        assert rel_rms(b.replica(f, r), fo) <= 1e-5, r
    b.close()


def test_bounded_wait_times_out_and_context_survives(oracle_mod):
    """A device wait that nothing satisfies (an mbarrier expecting bytes no
    copy delivers) gives up after its bound and reports LJ_ETIMEOUT; the
    context then computes correct forces again."""
    import time
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(6, 0.8442, 0.05, 1)
    s = lj.System(x, None, L)
    t0 = time.perf_counter()
    assert lj.lj_wait_selftest(s.ctx) == lj.LJ_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    s.check()                                   # the latch was cleared
    s.forces()
    s.check()
    fo = oracle_mod.forces_cells(x, L, mode=1)[0]
    f = s.f.double().cpu().numpy()[:, :3]
    assert np.sqrt(((f - fo) ** 2).sum() / (fo ** 2).sum()) <= 1e-5
    s.close()
