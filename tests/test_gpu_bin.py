"""GPU binning parity: cell ids, counts and starts bit-exact against the
oracle's serial counting sort; the order inside a cell is unspecified, so the
permutation is compared as one set per cell."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

from gpu_util import dense_cluster_state

pytestmark = pytest.mark.gpu


def _gpu_cells(x, L, precision="mixed", subdiv=1):
    from paper_0709_3225_gb300 import lj
    s = lj.System(x, None, L, precision=precision, cell_subdiv=subdiv)
    out = [t.cpu().numpy() for t in s.cells()]
    s.check()
    nc = s.ctx.nc
    s.close()
    return nc, out


def _compare(x, L, oracle_mod, precision="mixed", subdiv=1):
    nc, (cell_of, count, start, perm) = _gpu_cells(x, L, precision, subdiv)
    assert nc == oracle_mod.ncells(L, k=subdiv)
    o_cell, o_count, o_start, o_perm = oracle_mod.bin_cells(x, L, nc)
    assert np.array_equal(cell_of, o_cell)
    assert np.array_equal(count, o_count)
    assert np.array_equal(start, o_start)
    # same set of particles in every cell
    assert np.array_equal(np.sort(perm), np.arange(x.shape[0]))
    key = cell_of[perm].astype(np.int64) * (x.shape[0] + 1) + perm
    okey = o_cell[o_perm].astype(np.int64) * (x.shape[0] + 1) + o_perm
    assert np.array_equal(np.sort(key), np.sort(okey))
    assert np.array_equal(cell_of[perm], np.repeat(np.arange(nc ** 3), count))


def test_subdivision_two(oracle_mod):
    """Half-size cells (k = 2): the same exact binning rule with n = floor(2L/rc)."""
    x, L = inputs.jittered_fcc(9, 0.8442, 0.2, 5)
    _compare(x, L, oracle_mod, subdiv=2)
    _compare(inputs.uniform(1001, 7.0, 3), 7.0, oracle_mod, subdiv=2)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_fcc_2k(oracle_mod, precision):
    x, _, L, _ = inputs.workload_state("fluid-2k")
    _compare(x, L, oracle_mod, precision)


def test_jittered_131k(oracle_mod):
    x, L = inputs.jittered_fcc(32, 0.8442, 0.2, 5)
    _compare(x, L, oracle_mod)


@pytest.mark.parametrize("n", [1, 2, 31, 1000, 4097])
def test_uniform_ragged(oracle_mod, n):
    L = 12.3
    x = inputs.uniform(n, L, n) * 3.0 - L       # coordinates over three images
    _compare(x, L, oracle_mod)


def test_dense_cluster(oracle_mod):
    x, L = dense_cluster_state()
    _compare(x, L, oracle_mod)


def test_edge_coordinates(oracle_mod):
    L = 13.436769531060056
    nc = 5
    below = np.nextafter(L, 0.0)
    vals = [0.0, below, L, -1e-300, -0.0, -0.1, 2.5 * L, -3.3 * L, 1e9 + 0.3, -1e9 - 0.7,
            np.nextafter(0.0, 1.0)]
    vals += [k * (L / nc) for k in range(1, nc)]
    vals += [np.nextafter(k * (L / nc), 0.0) for k in range(1, nc)]
    vals += [np.nextafter(k * (L / nc), 1e300) for k in range(1, nc)]
    vals = np.array(vals)
    rng = np.random.default_rng(0)
    x = np.stack([vals, rng.permutation(vals), rng.permutation(vals)], axis=1)
    _compare(np.ascontiguousarray(x), L, oracle_mod)


def test_empty_system(oracle_mod):
    nc, (cell_of, count, start, perm) = _gpu_cells(np.zeros((0, 3)), 10.0)
    assert cell_of.size == 0 and perm.size == 0
    assert count.sum() == 0 and np.all(start == 0)


@pytest.mark.slow
def test_full_size_4m(oracle_mod):
    """Bit-exact binning at the 4,000,000-particle workload (jittered so that
    cells are uneven)."""
    x, L = inputs.jittered_fcc(100, 0.8442, 0.3, 11)
    _compare(x, L, oracle_mod)


@pytest.mark.parametrize("subdiv", [1, 2])
def test_deterministic_order_is_the_serial_counting_sort(oracle_mod, subdiv):
    """lj_set_deterministic: every cell's particles in index order, so the
    whole permutation equals the oracle's serial counting sort bit for bit."""
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(9, 0.8442, 0.2, 61)
    x[11, 0] = np.nan   # the extra cell is sorted too
    s = lj.System(x, None, L, cell_subdiv=subdiv)
    lj.lj_set_deterministic(s.ctx)
    cell_of, count, start, perm = (t.cpu().numpy() for t in s.cells())
    with pytest.raises(lj.LJError):
        s.check()
    good = np.isfinite(x).all(axis=1)
    nc = s.ctx.nc
    s.close()
    o_cell, o_count, o_start, o_perm = oracle_mod.bin_cells(np.ascontiguousarray(x[good]), L, nc)
    idx = np.flatnonzero(good)
    assert np.array_equal(perm[:good.sum()], idx[o_perm])
    assert perm[-1] == 11


def test_deterministic_forces_and_trajectories_repeat_bitwise():
    import torch
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(10, 0.8442, 0.1, 62)
    v = inputs.velocities(x.shape[0], 1.0, 62)
    runs = []
    for rep in range(2):
        s = lj.System(x, v, L)
        lj.lj_set_deterministic(s.ctx)
        lj.lj_set_graph(s.ctx)
        s.forces()
        f0 = s.f.clone()
        s.step(25)
        s.check()
        runs.append((f0, s.x.clone(), s.v.clone()))
        s.close()
    assert torch.equal(runs[0][0], runs[1][0])
    assert torch.equal(runs[0][1], runs[1][1]) and torch.equal(runs[0][2], runs[1][2])
