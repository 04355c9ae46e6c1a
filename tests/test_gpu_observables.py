"""Temperature and virial pressure on the GPU (lj_observables) against the
oracle's definitions (E_kin, E_pot, W from FP64 sums; T = 2 E_kin / (3N - 3),
P = (2 E_kin + W) / (3V)).

Tolerances: E_kin is an FP64 sum in another order (1e-12 relative), so T is
too; E_pot and W as in the force tests (mixed: 2e-6 of the sums of absolute
terms, FP64: 1e-11); P inherits W's bound divided by 3V."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"mixed": 2e-6, "fp64": 1e-11}


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("mode", [1, 2])
def test_observables_match_oracle(oracle_mod, precision, mode):
    from paper_0709_3225_gb300 import lj
    x, L = inputs.jittered_fcc(8, 0.8442, 0.1, 5)
    v = inputs.velocities(x.shape[0], 0.728, 6)
    s = lj.System(x, v, L, precision=precision, shift_mode=mode)
    o = s.observables()
    s.check()
    s.close()
    ref = oracle_mod.observables(x, v, L, mode=mode)
    _, ep, _, _ = oracle_mod.forces_cells(x, L, mode=mode)
    _, S = oracle_mod.stiffness(x, L, mode=mode)
    t = TOL[precision]
    assert o["e_kin"] == pytest.approx(ref["e_kin"], rel=1e-12)
    assert o["T"] == pytest.approx(ref["T"], rel=1e-12)
    assert o["T"] == pytest.approx(0.728, rel=1e-12)      # the velocities are rescaled to T exactly
    assert abs(o["e_pot"] - ref["e_pot"]) <= t * np.abs(ep).sum()
    wb = t * 0.5 * 2.5 * S.sum()
    assert abs(o["virial"] - ref["virial"]) <= wb
    assert abs(o["P"] - ref["P"]) <= wb / (3 * L ** 3) + 1e-12 * abs(ref["P"])
    assert o["e_tot"] == pytest.approx(o["e_kin"] + o["e_pot"], rel=1e-15, abs=1e-12)


def test_observables_ideal_gas_and_small_n(oracle_mod):
    from paper_0709_3225_gb300 import lj
    # eps = 0: W = 0 and P V = (2/3) E_kin exactly as the oracle pins it
    x, L = inputs.jittered_fcc(6, 0.8442, 0.1, 8)
    v = inputs.velocities(x.shape[0], 1.3, 9)
    s = lj.System(x, v, L, eps=0.0)
    o = s.observables()
    s.close()
    assert o["virial"] == 0.0 and o["e_pot"] == 0.0
    assert o["P"] * L ** 3 == pytest.approx(2.0 * o["e_kin"] / 3.0, rel=1e-12)
    # one particle: no degrees of freedom left after the momentum, T = 0
    x1 = np.array([[1.0, 2.0, 3.0]])
    s = lj.System(x1, np.array([[0.1, 0.2, 0.3]]), 9.0)
    o = s.observables()
    s.close()
    assert o["T"] == 0.0
    assert o["e_kin"] == pytest.approx(0.5 * 0.14, rel=1e-14)
