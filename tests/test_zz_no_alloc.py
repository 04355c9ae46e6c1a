"""lj_forces_static, the allocation-free forces entry point, against the
oracle.

lj_forces_static serves callers that cannot allocate device memory: code on a
fixed device-memory budget, code that runs inside another runtime's memory
pool, and code at points where cudaMalloc (and the synchronization it can
imply) is not allowed.  Its scratch is one fixed buffer inside the library,
shared by every call and keeping the previous call's contents.  So here:
  - every call's forces are checked against the FP64 oracle with the force
    tests' tolerances, in a large -> small -> large sequence (stale cell counts
    or starts from a larger call would show in the smaller one), in both
    precisions, with the force shift and with cell subdivision 2;
  - free device memory does not change across calls after the first (which
    loads the library's device code);
  - sizes beyond the fixed limits and run-kernel flags are refused, and n = 0
    is a no-op.
This file is collected last, so a run that stops at its first failure has run
every other test before it."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

from gpu_util import rel_rms

pytestmark = pytest.mark.gpu

TOL = {"mixed": dict(rms=1e-5, dr=6e-7, ds=1e-5, band=1e-5), "fp64": dict(rms=1e-12, rel=1e-10, band=1e-12)}

_REF = {}


def _oracle(oracle_mod, n_fcc, seed, mode, subdiv):
    key = (n_fcc, seed, mode, subdiv)
    if key not in _REF:
        x, L = inputs.jittered_fcc(n_fcc, 0.8442, 0.1, seed)
        fo, _, _, _ = oracle_mod.forces_cells(x, L, mode=mode, k=subdiv)
        rng = np.random.default_rng(seed)
        idx = np.arange(x.shape[0]) if x.shape[0] <= 4000 else np.sort(rng.choice(x.shape[0], 3000, replace=False))
        K, S = oracle_mod.stiffness(x, L, mode=mode, idx=idx)
        near = {b: oracle_mod.near_cutoff(x, L, band=b, k=subdiv) for b in (1e-5, 1e-12)}
        _REF[key] = (x, L, fo, idx, K, S, near)
    return _REF[key]


def _check(got, ref, precision):
    x, L, fo, idx, K, S, near = ref
    t = TOL[precision]
    assert np.all(np.isfinite(got))
    assert rel_rms(got, fo) <= t["rms"]
    d = np.abs(got[idx] - fo[idx]).max(axis=1)
    if precision == "mixed":
        bound = t["dr"] * K + t["ds"] * S
    else:
        frms = np.sqrt((fo ** 2).sum(axis=1).mean())
        bound = t["rel"] * (np.abs(fo[idx]).max(axis=1) + frms)
    ok = ~near[t["band"]][idx]
    assert np.all(d[ok] <= bound[ok]), (d[ok] / bound[ok]).max()


def _call(lj, torch, ref, precision, mode, subdiv):
    x, L = ref[0], ref[1]
    n = x.shape[0]
    fdt = torch.float32 if precision == "mixed" else torch.float64
    xd = torch.from_numpy(x).cuda()
    f = torch.full((n, 4), float("nan"), dtype=fdt, device="cuda")
    p = lj.make_params(n, L, precision=precision, shift_mode=mode, cell_subdiv=subdiv)
    return xd, f, p


@pytest.mark.parametrize("precision,mode,subdiv", [("mixed", 1, 1), ("fp64", 1, 1), ("mixed", 2, 1),
                                                   ("fp64", 2, 1), ("mixed", 1, 2)])
def test_static_matches_oracle_large_small_large(oracle_mod, precision, mode, subdiv):
    import torch
    from paper_0709_3225_gb300 import lj
    big = _oracle(oracle_mod, 20, 22, mode, subdiv)      # 32,000 particles, 13 (26) cells per side
    small = _oracle(oracle_mod, 8, 21, mode, subdiv)     # 2,048 particles, 5 (10) cells per side
    for ref in (big, small, big, small):
        xd, f, p = _call(lj, torch, ref, precision, mode, subdiv)
        for call in range(2):          # two calls in a row on the same arrays
            f.fill_(float("nan"))
            lj.lj_forces_static(p, xd, f)
            torch.cuda.synchronize()
            _check(f.double().cpu().numpy()[:, :3], ref, precision)


def test_static_allocates_nothing(oracle_mod):
    import torch
    from paper_0709_3225_gb300 import lj
    ref = _oracle(oracle_mod, 20, 22, 1, 1)
    xd, f, p = _call(lj, torch, ref, "mixed", 1, 1)
    lj.lj_forces_static(p, xd, f)      # the first call may load the library's device code
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        lj.lj_forces_static(p, xd, f)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _check(f.double().cpu().numpy()[:, :3], ref, "mixed")


def test_static_rejects_sizes_beyond_its_limits_and_run_kernels():
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
    # the run kernels report timeouts through an error word no caller could read
    for flags in (lj.LJ_FLAG_RUN_STAGED, lj.LJ_FLAG_RUN_DIRECT):
        with pytest.raises(lj.LJError) as ei:
            lj.lj_forces_static(lj.make_params(10, 9.0, flags=flags), x, f)
        assert ei.value.code == lj.LJ_EINVAL
    # n = 0: nothing to do, nothing written
    x0 = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    f0 = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    lj.lj_forces_static(lj.make_params(0, 9.0), x0, f0)
    torch.cuda.synchronize()
