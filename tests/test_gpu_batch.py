"""Batched ensembles: every replica of a batch gives what the oracle (and a
single-system context) gives for that replica alone; one cooperative launch
per step, graph-replayed or direct."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

from gpu_util import min_image, rel_rms

pytestmark = pytest.mark.gpu


def _small_ensemble(seed=5, nrep=6):
    e = inputs.ensemble(nrep, seed=seed, n_lo=500, n_hi=4000)
    xs, vs = inputs.ensemble_state(e)
    return e, xs, vs


@pytest.mark.parametrize("subdiv", [1, 2])
def test_batched_forces_match_oracle_and_single(oracle_mod, subdiv):
    """Cell subdivision 1 (27-cell stencil) and 2 (half-size cells, 125-cell
    stencil) in the batched kernel."""
    from paper_0709_3225_gb300 import lj
    e, xs, vs = _small_ensemble()
    b = lj.Batch(xs, vs, e.box, cell_subdiv=subdiv)
    b.forces()
    b.check()
    f = b.f.double().cpu().numpy()[:, :3]
    for r in range(b.nrep):
        fr = b.replica(f, r)
        fo = oracle_mod.forces_cells(xs[r], e.box[r], mode=1, k=subdiv)[0]
        assert rel_rms(fr, fo) <= 1e-5, r
        # the single-system per-particle bound over every particle of the
        # replica (those with a partner within 1e-5 of rc excepted)
        K, S = oracle_mod.stiffness(xs[r], e.box[r], mode=1)
        near = oracle_mod.near_cutoff(xs[r], e.box[r], band=1e-5)
        d = np.abs(fr - fo).max(axis=1)
        bound = 6e-7 * K + 1e-5 * S
        assert np.all(d[~near] <= bound[~near]), (r, (d[~near] / bound[~near]).max())
        # the same cell subdivision in a single-system context: the same pair
        # vectors, sums in another order
        s = lj.System(xs[r], None, e.box[r], cell_subdiv=subdiv)
        s.forces()
        assert rel_rms(fr, s.f.double().cpu().numpy()[:, :3]) <= 1e-6, r
        s.close()
    b.close()


@pytest.mark.parametrize("use_graph,mode,subdiv", [(True, 1, 1), (True, 2, 1), (False, 1, 1), (False, 2, 1),
                                                  (True, 2, 2), (False, 1, 2)])
def test_batched_steps_match_oracle(oracle_mod, use_graph, mode, subdiv):
    """23 steps.  With the force-shifted potential the force is continuous
    and positions agree to FP32 rounding; with the energy shift a pair whose
    distance is within rounding of rc may be counted on either side, and one
    such event moves a particle by ~dt^2 F(rc) per step afterwards, so the
    bound allows 1e-4 for single particles and checks the RMS tightly."""
    from paper_0709_3225_gb300 import lj
    e, xs, vs = _small_ensemble(seed=7, nrep=5)
    b = lj.Batch(xs, vs, e.box, shift_mode=mode, cell_subdiv=subdiv)
    b.set_tuning(cells_per_grab=2, use_graph=use_graph)
    b.step(8)
    b.step(12)
    b.check()
    n0, _ = b.launches()
    b.step(3)
    n1, graph = b.launches()
    assert n1 - n0 == 4                      # one launch per step + the closing kick
    assert graph == use_graph
    x = b.x.cpu().numpy()
    for r in range(b.nrep):
        xo, vo = xs[r].copy(), vs[r].copy()
        fo = oracle_mod.forces_cells(xo, e.box[r], mode=mode)[0]
        # a force error of RMS 1e-5 F_rms, integrated over n steps, moves
        # positions by at most ~ dt^2 n^2 / 2 of it
        drift = 0.5 * 0.005 ** 2 * 23 ** 2 * 1e-5 * np.sqrt((fo ** 2).sum(axis=1).mean())
        oracle_mod.vv(xo, vo, fo, e.box[r], 23, mode=mode)
        d = np.abs(min_image(b.replica(x, r) - xo, e.box[r]))
        assert np.sqrt((d ** 2).mean()) <= drift, (r, drift)
        assert d.max() <= (20 * drift if mode == 2 else 1e-4), r
    b.close()


def test_batched_energy_and_relaxation(oracle_mod):
    from paper_0709_3225_gb300 import lj
    e, xs, vs = _small_ensemble(seed=9, nrep=4)
    b = lj.Batch(xs, vs, e.box)
    en = b.energy()
    for r in range(b.nrep):
        _, ep, eo, _ = oracle_mod.forces_cells(xs[r], e.box[r], mode=1)
        assert en[r, 0] == pytest.approx(oracle_mod.ekin(vs[r]), rel=1e-12)
        assert abs(en[r, 1] - eo) <= 2e-6 * np.abs(ep).sum()
    # 50 capped steepest-descent steps, against the oracle's relaxation
    b.relax(50, 1e-3, 0.05)
    b.check()
    x = b.x.cpu().numpy()
    en2 = b.energy()
    for r in range(b.nrep):
        xo, _ = oracle_mod.relax(xs[r], e.box[r], 50, alpha=1e-3, dmax=0.05)
        # n steps of x += alpha F move a force error of RMS 1e-5 F_rms by n alpha
        f0 = oracle_mod.forces_cells(xs[r], e.box[r], mode=1)[0]
        drift = 50 * 1e-3 * 1e-5 * np.sqrt((f0 ** 2).sum(axis=1).mean())
        d = np.abs(min_image(b.replica(x, r) - xo, e.box[r]))
        assert np.sqrt((d ** 2).mean()) <= drift, (r, drift)
        assert d.max() <= 50 * drift, r
        assert en2[r, 1] < en[r, 1]
    b.close()


def test_tuning_knobs_give_same_forces():
    from paper_0709_3225_gb300 import lj
    e, xs, vs = _small_ensemble(seed=11, nrep=3)
    b = lj.Batch(xs, vs, e.box)
    b.forces()
    ref = b.f.clone()
    rms = float(ref[:, :3].double().pow(2).sum(dim=1).mean().sqrt())
    for cpg, gw in ((1, 0), (16, 32), (3, 16), (2, 2), (5, 4), (4, -1)):
        b.set_tuning(cells_per_grab=cpg, use_graph=True, group_width=gw)
        b.forces()
        # same arithmetic up to the order of FP32 sums
        diff = (b.f[:, :3] - ref[:, :3]).double().abs()
        assert bool((diff <= 1e-5 * (ref[:, :3].double().abs() + rms)).all())
    b.check()
    b.close()


@pytest.mark.slow
def test_full_ensemble_256(oracle_mod):
    """The 256-replica ensemble (N_r in [500, 50000]): forces of sampled
    particles in sampled replicas against the oracle's per-particle
    definition, with the single-system per-particle bound (no extra slack);
    10 graph-replayed steps without latched errors."""
    from paper_0709_3225_gb300 import lj
    e = inputs.ensemble()
    xs, vs = inputs.ensemble_state(e)
    b = lj.Batch(xs, vs, e.box)
    b.forces()
    b.check()
    f = b.f.double().cpu().numpy()
    rng = np.random.default_rng(0)
    for r in rng.choice(b.nrep, 6, replace=False):
        fr = b.replica(f, r)
        near = oracle_mod.near_cutoff(xs[r], e.box[r], band=1e-5)
        for i in rng.choice(xs[r].shape[0], 8, replace=False):
            if near[i]:
                continue        # a partner within FP32 rounding of rc may count on either side
            fi, _ = oracle_mod.force_one(xs[r], e.box[r], int(i))
            K, S = oracle_mod.stiffness(xs[r], e.box[r], idx=[int(i)])
            assert np.abs(fr[i, :3] - fi).max() <= 6e-7 * K[0] + 1e-5 * S[0]
    b.step(10)
    b.check()
    b.close()


def test_batch_rejects_bad_subdivision():
    from paper_0709_3225_gb300 import lj
    e, xs, vs = _small_ensemble(seed=13, nrep=2)
    with pytest.raises(lj.LJError) as ei:
        lj.Batch(xs, vs, e.box, cell_subdiv=3)
    assert ei.value.code == lj.LJ_EINVAL


@pytest.mark.parametrize("mode", [1, 2])
def test_pair_once_and_27_cell_batch_kernels(oracle_mod, mode):
    """The batch's two force kernels (7: each pair once, the default; 3: the
    27-cell code) against the oracle per replica, and 15 steps of each against
    the oracle's trajectory."""
    from paper_0709_3225_gb300 import lj
    e, xs, vs = _small_ensemble(seed=17, nrep=4)
    for kernel in (7, 3):
        b = lj.Batch(xs, vs, e.box, shift_mode=mode)
        b.set_kernel(kernel)
        b.forces(energy=True)
        b.check()
        f = b.f.double().cpu().numpy()
        for r in range(b.nrep):
            fo, epo, _, _ = oracle_mod.forces_cells(xs[r], e.box[r], mode=mode)
            fr = b.replica(f, r)
            assert rel_rms(fr[:, :3], fo) <= 1e-5, (kernel, r)
            K, S = oracle_mod.stiffness(xs[r], e.box[r], mode=mode)
            near = oracle_mod.near_cutoff(xs[r], e.box[r], band=1e-5)
            d = np.abs(fr[:, :3] - fo).max(axis=1)
            assert np.all(d[~near] <= (6e-7 * K + 1e-5 * S)[~near]), (kernel, r)
            assert np.all(np.abs(fr[~near, 3] - epo[~near]) <= 1e-5 * np.abs(epo).max()), (kernel, r)
        b.step(15)
        b.check()
        x = b.x.cpu().numpy()
        for r in range(b.nrep):
            xo, vo = xs[r].copy(), vs[r].copy()
            fo = oracle_mod.forces_cells(xo, e.box[r], mode=mode)[0]
            # a force error of RMS 1e-5 F_rms moves positions by at most
            # ~ dt^2 n^2 / 2 of it over n steps (as in the trajectory test above)
            drift = 0.5 * 0.005 ** 2 * 15 ** 2 * 1e-5 * np.sqrt((fo ** 2).sum(axis=1).mean())
            oracle_mod.vv(xo, vo, fo, e.box[r], 15, mode=mode)
            d = np.abs(min_image(b.replica(x, r) - xo, e.box[r]))
            assert np.sqrt((d ** 2).mean()) <= drift, (kernel, r)
        b.close()


def test_batch_kernel_choice_is_checked():
    from paper_0709_3225_gb300 import lj
    e, xs, vs = _small_ensemble(seed=19, nrep=2)
    b = lj.Batch(xs, vs, e.box)
    with pytest.raises(lj.LJError):
        b.set_kernel(5)
    b.close()
    b2 = lj.Batch(xs, vs, e.box, cell_subdiv=2)
    with pytest.raises(lj.LJError):
        b2.set_kernel(7)
    b2.set_kernel(3)
    b2.close()
