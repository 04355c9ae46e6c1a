"""lj_forces_static, the allocation-free forces entry point, against the
context-based lj_forces.

lj_forces_static serves callers that cannot allocate device memory (a fixed
memory budget, another runtime's pool, places where cudaMalloc is not
allowed): its scratch is a fixed buffer inside the library.  Here it must
give, on two calls in a row, the forces lj_forces gives, within the force
tests' tolerances, and refuse sizes beyond its limits."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

from gpu_util import rel_rms

pytestmark = pytest.mark.gpu

TOL = {"mixed": dict(rms=1e-5, dr=6e-7, ds=1e-5), "fp64": dict(rms=1e-12, rel=1e-10)}


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("n_fcc,seed", [(8, 21), (20, 22)])
def test_static_matches_lj_forces(oracle_mod, precision, n_fcc, seed):
    import torch
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(n_fcc, 0.8442, 0.1, seed)
    ref = lj.System(x, None, L, precision=precision)
    ref.forces()
    ref.check()
    f_ref = ref.f.double().cpu().numpy()[:, :3]
    params = lj.make_params(x.shape[0], L, precision=precision)
    xd = ref.x
    t = TOL[precision]
    near = oracle_mod.near_cutoff(x, L, band=1e-5 if precision == "mixed" else 1e-12)
    if precision == "mixed":
        K, S = oracle_mod.stiffness(x, L)
        bound = t["dr"] * K + t["ds"] * S
    else:
        bound = t["rel"] * (np.abs(f_ref).max(axis=1) + np.sqrt((f_ref ** 2).sum(axis=1).mean()))
    for call in range(2):
        f = torch.full((x.shape[0], 4), float("nan"), dtype=ref.f.dtype, device=xd.device)
        lj.lj_forces_static(params, xd, f)
        torch.cuda.synchronize()
        got = f.double().cpu().numpy()[:, :3]
        assert np.all(np.isfinite(got)), call
        assert rel_rms(got, f_ref) <= t["rms"], call
        d = np.abs(got - f_ref).max(axis=1)
        assert np.all(d[~near] <= bound[~near]), call
    ref.close()


def test_static_rejects_sizes_beyond_its_limits():
    import torch
    from paper_0709_3225_gb300 import lj
    n = lj.LJ_STATIC_MAX_N + 1
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(lj.LJError) as ei:
        lj.lj_forces_static(lj.make_params(n, 60.0), x, f)
    assert ei.value.code == lj.LJ_EOVERFLOW
    # 33 cells per side is over the cell limit even for a small particle count
    x = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(lj.LJError) as ei:
        lj.lj_forces_static(lj.make_params(10, 33 * 2.5 + 0.1), x, f)
    assert ei.value.code == lj.LJ_EOVERFLOW
