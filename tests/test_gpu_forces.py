"""GPU force parity against the FP64 oracle (Section 2 pair force over the
Section 3 cell list).

Tolerances (derived from the arithmetic):
  mixed: relative RMS force error <= 1e-5 over all particles; per particle
         and component |df_i| <= 6e-7 K_i + 1e-5 S_i, where K_i = sum_j
         (|F'(r_ij)| + |F(r_ij)|/r_ij) and S_i = sum_j |F(r_ij)| (FP32
         rounding of the pair vectors, <= 6e-7 sigma, and of a sum of <= ~100
         terms), for particles with no partner within 1e-5 of rc; energy and
         virial (FP64 sums of FP32 terms) to 2e-6 relative.
  fp64:  per particle |df| <= 1e-10 (|f| + f_rms), energy / virial to 1e-11.
A pair whose distance is within working precision of rc may fall on either
side of the cutoff: such particles are excluded from the per-particle bound
(and stay in the RMS)."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

from gpu_util import dense_cluster_state, rel_rms

pytestmark = pytest.mark.gpu

TOL = {"mixed": dict(rms=1e-5, dr=6e-7, ds=1e-5, e=2e-6, band=1e-5),
       "fp64": dict(rms=1e-12, rel=1e-10, e=1e-11, band=1e-12)}


def _gpu_forces(x, L, precision, mode=1, flags=0, eps=1.0, sigma=1.0, rc=2.5, subdiv=1, gw=None, kernel=None,
                grab=4):
    from paper_0709_3225_gb300 import lj
    s = lj.System(x, None, L, precision=precision, shift_mode=mode, flags=flags, eps=eps, sigma=sigma, rc=rc,
                  cell_subdiv=subdiv)
    if gw is not None or kernel is not None:
        lj.lj_set_tuning(s.ctx, 3 if kernel is None else kernel, gw or 0, grab)
    e, w = s.forces(energy=True)
    f = s.f.double().cpu().numpy()
    s.check()
    s.close()
    return f, e, w


def _check(x, L, oracle_mod, precision, mode=1, flags=0, eps=1.0, sigma=1.0, rc=2.5, subdiv=1, gw=None,
           kernel=None, grab=4):
    f, e, w = _gpu_forces(x, L, precision, mode, flags, eps, sigma, rc, subdiv, gw, kernel, grab)
    fo, epo, eo, wo = oracle_mod.forces_cells(x, L, eps=eps, sigma=sigma, rc=rc, mode=mode, k=subdiv)
    t = TOL[precision]
    near = oracle_mod.near_cutoff(x, L, rc=rc, band=t["band"])
    assert rel_rms(f[:, :3], fo) <= t["rms"]
    d = np.abs(f[:, :3] - fo).max(axis=1)
    frms = np.sqrt((fo ** 2).sum(axis=1).mean()) if fo.size else 0.0
    K, S = oracle_mod.stiffness(x, L, eps=eps, sigma=sigma, rc=rc, mode=mode)
    if precision == "mixed":
        bound = t["dr"] * K + t["ds"] * S
        assert np.all(d[~near] <= bound[~near]), (d[~near] / bound[~near]).max()
    else:
        bound = t["rel"] * (np.abs(fo).max(axis=1) + frms)
        assert np.all(d[~near] <= bound[~near])
    # Energy and virial: relative to the sums of absolute terms (the signed
    # sums can nearly cancel): sum_i |e_i| and sum_pairs r|F| <= rc/2 sum_i S_i.
    assert abs(e - eo) <= t["e"] * max(np.abs(epo).sum(), 1e-300) + 1e-12
    assert abs(w - wo) <= t["e"] * 0.5 * rc * S.sum() + 1e-12
    # per-particle energies in f[:, 3]
    escale = np.abs(epo).max() if epo.size else 1.0
    assert np.all(np.abs(f[~near, 3] - epo[~near]) <= (1e-5 if precision == "mixed" else 1e-10) * escale)
    return f, fo


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_liquid_2k(oracle_mod, precision, mode):
    x, L = inputs.jittered_fcc(8, 0.8442, 0.1, 1)
    _check(x, L, oracle_mod, precision, mode)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("kernel", [3, 7])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("state", ["liquid", "dense", "rho095", "cluster", "three_cells", "dilute"])
def test_pairs_once_and_27_cell_kernels(oracle_mod, precision, kernel, mode, state):
    """The kernels that evaluate each pair once (Newton's third law, half
    stencil, kernel 7) and the 27-cell kernels (3), FP32-mixed and FP64,
    against the oracle: a liquid; rho = 2 (cells of ~32 particles: the
    four-group layout and more than 32 home particles per pass; FP64 lists
    in several batches); rho = 0.95 (cells over 16); a dense blob in a
    dilute gas (the plain path of cells whose half stencil overflows the
    slice); 3 cells per side; a dilute gas."""
    if state == "liquid":
        x, L = inputs.jittered_fcc(8, 0.8442, 0.1, 61)
    elif state == "dense":
        x, L = inputs.jittered_fcc(8, 2.0, 0.05, 62)
    elif state == "rho095":
        x, L = inputs.jittered_fcc(9, 0.95, 0.1, 63)
    elif state == "cluster":
        x, L = dense_cluster_state(64)
    elif state == "three_cells":
        x, L = inputs.jittered_fcc(5, 0.8442, 0.1, 65)
    else:
        x, L = inputs.jittered_fcc(7, 0.2, 0.2, 66)
    for grab in (0, 4):
        _check(x, L, oracle_mod, precision, mode, kernel=kernel, grab=grab)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("flags", [0, 1, 2])
def test_kernel_variants(oracle_mod, precision, flags):
    """Warp-per-cell kernel, run kernel with bulk-copy staging and run kernel
    with direct global reads give the same forces."""
    x, L = inputs.jittered_fcc(10, 0.8442, 0.1, 2)
    _check(x, L, oracle_mod, precision, 1, flags)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_subdivision_two(oracle_mod, mode):
    """Cell subdivision k = 2: half-size cells, 125-cell stencil, same forces
    as the oracle's k = 2 cell list (itself equal to k = 1)."""
    x, L = inputs.jittered_fcc(8, 0.8442, 0.1, 21)
    _check(x, L, oracle_mod, "mixed", mode, subdiv=2)


@pytest.mark.parametrize("subdiv", [1, 2])
@pytest.mark.parametrize("gw", [0, -1, 2, 4, 8, 16, 32])
def test_group_widths(oracle_mod, subdiv, gw):
    """Every lane-group width (chunks of gw home particles, 32 / gw candidate
    streams; 0 the compiled-in default, -1 chosen per cell) gives the
    oracle's forces."""
    x, L = inputs.jittered_fcc(7, 0.8442, 0.12, 30 + gw)
    _check(x, L, oracle_mod, "mixed", 1, subdiv=subdiv, gw=gw)


@pytest.mark.parametrize("n_fcc,rho", [(4, 0.8442), (5, 0.8442), (4, 0.3), (9, 0.95)])
def test_subdivision_two_box_sizes(oracle_mod, n_fcc, rho):
    """5, 6, 7 ... half-size cells per side: stencil windows that wrap onto
    themselves (5 cells), sparse and dense cells."""
    x, L = inputs.jittered_fcc(n_fcc, rho, 0.08, n_fcc + 40)
    _check(x, L, oracle_mod, "mixed", subdiv=2)


@pytest.mark.parametrize("n_fcc,rho", [(5, 0.8442), (6, 0.8442), (7, 0.5), (9, 0.95), (12, 0.8442), (4, 0.3)])
def test_box_sizes(oracle_mod, n_fcc, rho):
    """3, 4, 5 ... cells per side: windows that wrap on both sides; sparse
    cells (8-lane groups)."""
    x, L = inputs.jittered_fcc(n_fcc, rho, 0.08, n_fcc)
    for flags in (0, 1):
        _check(x, L, oracle_mod, "mixed", flags=flags)
    _check(x, L, oracle_mod, "fp64")


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("flags", [0, 1])
def test_dense_cluster_and_overflow(oracle_mod, precision, flags):
    """Cells with > 32 particles (several passes / plain path) and stencil
    windows larger than the staging capacity (global-memory fallback)."""
    x, L = dense_cluster_state()
    _check(x, L, oracle_mod, precision, flags=flags)
    if precision == "mixed" and flags == 0:
        _check(x, L, oracle_mod, precision, subdiv=2)
        for gw in (2, 32):
            _check(x, L, oracle_mod, precision, gw=gw)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_fp64_pair_lists_in_batches(oracle_mod, mode):
    """FP64 warp kernel: a dense liquid (rho 1.1) with rc = 3, so a home
    cell's in-range pair lists (~30 particles x ~120 partners) exceed one
    list batch and are taken in several; the same forces as the oracle and
    as the FP64 run kernel."""
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(8, 1.1, 0.05, 50 + mode)
    f, _ = _check(x, L, oracle_mod, "fp64", mode, rc=3.0)
    _check(x, L, oracle_mod, "fp64", mode, rc=3.0, kernel=7)
    s = lj.System(x, None, L, precision="fp64", shift_mode=mode, rc=3.0)
    lj.lj_set_tuning(s.ctx, 1)
    e, w = s.forces(energy=True)
    fr = s.f.cpu().numpy()
    s.check()
    s.close()
    assert np.abs(fr - f).max() <= 1e-13 * np.abs(f).max()


@pytest.mark.parametrize("first", [3, 7])
@pytest.mark.parametrize("grab,mode", [(0, 1), (1, 1), (4, 1), (4, 0), (4, 2)])
def test_fp64_kernels_agree(first, grab, mode):
    """FP64 warp kernels (27-cell or pair-once; static striding or work
    pulls) against the run kernel, on a liquid with empty, sparse and
    crowded cells."""
    from paper_0709_3225_gb300 import lj
    x, L = dense_cluster_state(seed=7)
    out = []
    for kernel in (first, 1):
        s = lj.System(x, None, L, precision="fp64", shift_mode=mode)
        lj.lj_set_tuning(s.ctx, kernel, 0, grab)
        e, w = s.forces(energy=True)
        out.append((s.f.cpu().numpy(), e, w))
        s.check()
        s.close()
    (fa, ea, wa), (fb, eb, wb) = out
    # both at FP64 accuracy: Newton-refined reciprocals against IEEE division,
    # different summation orders
    assert np.abs(fa - fb).max() <= 1e-13 * np.abs(fb).max()
    assert ea == pytest.approx(eb, rel=1e-13) and wa == pytest.approx(wb, rel=1e-13)


def test_ragged_random_gas(oracle_mod):
    # Uniform random gas with a minimum-distance filter: empty cells, uneven
    # counts, particle count not a multiple of anything.
    L = 15.1
    x = inputs.uniform(3000, L, 9)
    keep = [0]
    for i in range(1, x.shape[0]):
        d = x[keep] - x[i]
        d -= L * np.round(d / L)
        if (d * d).sum(axis=1).min() > 0.8 ** 2:
            keep.append(i)
    x = np.ascontiguousarray(x[keep])
    _check(x, L, oracle_mod, "mixed")
    _check(x, L, oracle_mod, "fp64")


@pytest.mark.parametrize("eps,sigma,rc", [(0.9, 1.05, 2.5), (1.3, 0.9, 3.0)])
def test_other_parameters(oracle_mod, eps, sigma, rc):
    x, L = inputs.jittered_fcc(8, 0.8442, 0.08, 4)
    for mode in (1, 2):
        _check(x, L, oracle_mod, "mixed", mode, eps=eps, sigma=sigma, rc=rc)
        _check(x, L, oracle_mod, "fp64", mode, eps=eps, sigma=sigma, rc=rc)


def test_translation_invariance_gpu(oracle_mod):
    x, L = inputs.jittered_fcc(8, 0.8442, 0.08, 6)
    f1, _, _ = _gpu_forces(x, L, "fp64")
    f2, _, _ = _gpu_forces(x + np.array([5.5, -100.25, 33.0]), L, "fp64")
    assert np.abs(f1[:, :3] - f2[:, :3]).max() <= 1e-9 * np.abs(f1).max()


def test_fcc_lattice_forces_vanish():
    x, _, L, _ = inputs.workload_state("fluid-2k")
    f, e, w = _gpu_forces(x, L, "fp64")
    assert np.abs(f[:, :3]).max() < 1e-10
    f, e, w = _gpu_forces(x, L, "mixed")
    assert np.abs(f[:, :3]).max() < 1e-3


@pytest.mark.slow
def test_liquid_131k(oracle_mod):
    x, L = inputs.jittered_fcc(32, 0.8442, 0.1, 8)
    _check(x, L, oracle_mod, "mixed")
    _check(x, L, oracle_mod, "fp64")


@pytest.mark.slow
@pytest.mark.parametrize("precision,subdiv", [("mixed", 1), ("fp64", 1), ("mixed", 2)])
def test_full_size_4m_sampled(oracle_mod, precision, subdiv):
    """The 4,000,000-particle workload in the launch configuration the
    benchmark uses: 256 sampled particles against the oracle's per-particle
    definition, plus zero net force (Newton III) over all particles."""
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(100, 0.8442, 0.1, 12)
    s = lj.System(x, None, L, precision=precision, cell_subdiv=subdiv)
    s.forces()
    s.check()
    f = s.f.double().cpu().numpy()
    s.close()
    idx = np.random.default_rng(0).choice(x.shape[0], 256, replace=False)
    ref = np.array([oracle_mod.force_one(x, L, int(i))[0] for i in idx])
    got = f[idx, :3]
    err = np.abs(got - ref).max(axis=1)
    if precision == "mixed":
        K, S = oracle_mod.stiffness(x, L, idx=idx)
        bound = 6e-7 * K + 1e-5 * S
    else:
        bound = 1e-9 * (np.abs(ref).max() + 1)
    bad = err > bound
    # any sampled particle over the bound must have a pair at the cutoff
    for i in np.flatnonzero(bad):
        fi, _ = oracle_mod.force_one(x, L, int(idx[i]))
        d = x - x[idx[i]]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(axis=1))
        assert np.any(np.abs(r - 2.5) < 1e-5), (i, err[i])
    assert rel_rms(got, ref) <= (1e-5 if precision == "mixed" else 1e-12)
    # Newton III: pair terms cancel up to rounding (random-walk bound).
    frms = float(np.sqrt((ref ** 2).sum(axis=1).mean()))
    net = np.abs(f[:, :3].sum(axis=0)).max()
    unit = 1e-5 if precision == "mixed" else 1e-14
    assert net <= 10 * np.sqrt(x.shape[0]) * unit * frms


@pytest.mark.parametrize("gw", [0, 2, 4, 16, 32])
def test_bulk_copied_stencils(oracle_mod, gw):
    """Kernel 5 (each cell's stencil bulk-copied into shared memory while the
    previous cell computes) gives the oracle's forces, including cells that
    take its plain path (dense cluster) and every lane-group width."""
    from paper_0709_3225_gb300 import lj
    for x, L in (inputs.jittered_fcc(9, 0.8442, 0.12, 200 + gw), dense_cluster_state(4)):
        s = lj.System(x, None, L)
        lj.lj_set_tuning(s.ctx, 5, gw, 4)
        e, w = s.forces(energy=True)
        s.check()
        f = s.f.double().cpu().numpy()
        s.close()
        fo, epo, eo, wo = oracle_mod.forces_cells(x, L, mode=1)
        near = oracle_mod.near_cutoff(x, L, band=1e-5)
        K, S = oracle_mod.stiffness(x, L, mode=1)
        d = np.abs(f[:, :3] - fo).max(axis=1)
        assert rel_rms(f[:, :3], fo) <= 1e-5
        assert np.all(d[~near] <= (6e-7 * K + 1e-5 * S)[~near])
        assert abs(e - eo) <= 2e-6 * np.abs(epo).sum() + 1e-12


def _cutoff_pairs(delta):
    """Isolated pairs at separations rc (1 - delta) and rc (1 + delta) along
    axis, face-diagonal and body-diagonal directions, centred on a 3 x 3 x 3
    grid whose first plane in each axis sits on the periodic boundary (those
    pairs straddle it), in a box of 8 cells per side; every particle of one
    pair is more than 4 sigma from those of the others."""
    L, rc = 20.0, 2.5
    dirs = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, -1, 1], [1, 1, 1], [-1, 1, -1]], float)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    sites = np.stack(np.meshgrid(*[np.arange(3)] * 3, indexing="ij"), -1).reshape(-1, 3) * (L / 3.0)
    x, inside = [], []
    for q, base in enumerate(sites):
        u = dirs[q % len(dirs)]
        r = rc * (1.0 - delta) if q % 2 == 0 else rc * (1.0 + delta)
        x += [base - 0.5 * r * u, base + 0.5 * r * u]
        inside += [r < rc, r < rc]
    x = np.array(x) % L
    return np.ascontiguousarray(x), L, np.array(inside)


@pytest.mark.parametrize("precision,kernel", [("mixed", None), ("mixed", 3), ("fp64", None)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_cutoff_decision_at_rc(oracle_mod, precision, kernel, mode):
    # r^2 < rc^2 decides a pair (strict cutoff, Section 2).  Pairs 2e-6 rc
    # inside the cutoff feel their pair force; pairs 2e-6 rc outside feel
    # nothing at all (the FP32 rounding of r^2 is ~1e-7 relative, far below
    # the 4e-6 between the two sides).
    x, L, inside = _cutoff_pairs(2e-6)
    f, _, _ = _gpu_forces(x, L, precision, mode, kernel=kernel)
    fo, _, _, _ = oracle_mod.forces_brute(x, L, mode=mode)
    assert np.all(f[~inside, :3] == 0.0)
    assert np.all(np.abs(fo[~inside]) == 0.0)
    fin, foin = f[inside, :3], fo[inside]
    if mode != 2:   # the force-shifted force nearly vanishes at rc
        assert np.all(np.linalg.norm(foin, axis=1) > 0.03)
    d = np.abs(fin - foin).max(axis=1)
    if precision == "mixed":   # the per-particle bound of the other parity tests
        K, S = oracle_mod.stiffness(x, L, mode=mode)
        bound = TOL["mixed"]["dr"] * K[inside] + TOL["mixed"]["ds"] * S[inside]
    else:
        bound = TOL["fp64"]["rel"] * (np.abs(foin).max(axis=1) + 1e-3)
    assert np.all(d <= bound), (d / bound).max()
