"""Pins of the oracle's cell grid and binning (Section 3 and the worked
example of Section 3.2)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cell_grid_example.txt")


def _golden():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def test_paper_worked_example(oracle_mod):
    g = _golden()
    n = oracle_mod.ncells(g["L"], g["rc"])
    assert n == int(g["n_x"])
    assert g["L"] / n == pytest.approx(g["cell_side"])
    assert g["L"] / n / g["rc"] - 1 == pytest.approx(g["cell_growth"])


def test_paper_growth_ratios_from_binning(oracle_mod):
    """A 10% larger cell holds ~33% more particles and gives ~77% more
    candidate interactions over the 27-cell stencil (Section 3.2): measured
    on uniform random systems binned by the oracle."""
    g = _golden()
    rho = 1.0
    occ, inter = [], []
    for side in (g["rc"], g["cell_side"]):
        L = 4 * side
        n = int(round(rho * L ** 3))
        o_s, i_s = [], []
        for seed in range(8):
            x = inputs.uniform(n, L, seed)
            _, count, _, _ = oracle_mod.bin_cells(x, L, 4)
            cnt = count.reshape(4, 4, 4)
            nb = sum(np.roll(cnt, (a, b, c), axis=(0, 1, 2))
                     for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
            o_s.append(count.mean())
            i_s.append(float((cnt * nb).sum()))
        occ.append(np.mean(o_s))
        inter.append(np.mean(i_s))
    assert occ[1] / occ[0] - 1 == pytest.approx(g["particles_per_cell_growth"], abs=0.01)
    assert inter[1] / inter[0] - 1 == pytest.approx(g["interactions_growth"], abs=0.03)


def test_paper_occupancy_at_unit_density(oracle_mod):
    g = _golden()
    L = 10 * g["rc"]
    n = int(round(g["rho_occupancy"] * L ** 3))
    x = inputs.uniform(n, L, 3)
    nc = oracle_mod.ncells(L, g["rc"])
    _, count, _, _ = oracle_mod.bin_cells(x, L, nc)
    assert count.mean() == pytest.approx(g["occupancy_per_cell"], rel=0.03)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_ncells_floor_rule(oracle_mod, k):
    for L in [7.5, 7.6, 8.4, 13.43677, 53.74708, 167.95962]:
        n = oracle_mod.ncells(L, 2.5, k)
        assert n * 2.5 / k <= L + 1e-12 < (n + 1) * 2.5 / k


def _check_csr(cell_of, count, start, perm, n, ncell):
    assert count.sum() == n
    assert np.array_equal(np.bincount(cell_of, minlength=ncell), count)
    assert start[0] == 0 and start[-1] == n
    assert np.array_equal(np.diff(start), count)
    assert np.array_equal(np.sort(perm), np.arange(n))
    for c in np.flatnonzero(count)[:2000]:
        sl = perm[start[c]:start[c + 1]]
        assert np.all(cell_of[sl] == c)
        assert np.all(np.diff(sl) > 0)


@pytest.mark.parametrize("n,L,nc", [(1000, 10.0, 4), (5000, 16.8, 6), (777, 9.1, 3)])
def test_binning_against_interval_geometry(oracle_mod, n, L, nc):
    """Each particle's cell satisfies c * L/nc <= w < (c+1) * L/nc, checked
    in exact rational arithmetic on positions away from cell faces."""
    rng = np.random.default_rng(n)
    x = rng.random((n, 3)) * 3 * L - L          # three periodic images
    cell_of, count, start, perm = oracle_mod.bin_cells(x, L, nc)
    _check_csr(cell_of, count, start, perm, n, nc ** 3)
    cz, rem = np.divmod(cell_of, nc * nc)
    cy, cx = np.divmod(rem, nc)
    cc = np.stack([cx, cy, cz], axis=1)
    Lq = Fraction(L)
    side = Lq / nc
    checked = 0
    for i in range(0, n, 7):
        for d in range(3):
            xq = Fraction(float(x[i, d]))
            w = xq - Lq * ((xq / Lq).__floor__())
            c = int(cc[i, d])
            lo, hi = c * side, (c + 1) * side
            if min(abs(w - lo), abs(w - hi)) < Fraction(1, 10 ** 9):
                continue
            assert lo <= w < hi
            checked += 1
    assert checked > n // 3


def test_binning_edge_cases(oracle_mod):
    L = 13.436769531060056
    nc = 5
    below = np.nextafter(L, 0.0)
    faces = [k * (L / nc) for k in range(1, nc)]
    xs = [0.0, below, L, -1e-300, -0.1, 2.5 * L, -3.3 * L] + faces
    x = np.array([[v, 0.5, 0.5] for v in xs])
    cell_of, count, start, perm = oracle_mod.bin_cells(x, L, nc)
    cx = cell_of % nc
    assert cx[0] == 0                 # x = 0
    assert cx[1] == nc - 1            # x = L - ulp: clamped into the last cell
    assert cx[2] == 0                 # x = L wraps to 0
    assert cx[3] == 0                 # tiny negative wraps up to L, then back to 0
    assert cx[4] == nc - 1            # -0.1 wraps to L - 0.1
    assert cx[5] == int(0.5 * nc)     # 2.5 L wraps to L/2
    # Faces: the chosen cell is one of the two cells that share the face.
    for k, c in zip(range(1, nc), cx[7:]):
        assert c in (k - 1, k)
    _check_csr(cell_of, count, start, perm, len(xs), nc ** 3)


def test_binning_empty(oracle_mod):
    cell_of, count, start, perm = oracle_mod.bin_cells(np.zeros((0, 3)), 10.0, 4)
    assert count.sum() == 0 and np.all(start == 0) and perm.size == 0
