"""Checkpoint files on the host: what is written is read back unchanged, and
files that do not describe a run of the stated parameters are refused."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import lj


def _state(n=40, precision="mixed", seed=1):
    rng = np.random.default_rng(seed)
    p = lj.make_params(n, 9.0, eps=0.9, sigma=1.05, rc=2.5, dt=0.004, mass=1.5, shift_mode=lj.LJ_SHIFT_FORCE,
                       precision=precision, cell_subdiv=1, flags=0)
    x = rng.uniform(0.0, 9.0, (n, 3))
    v = rng.normal(size=(n, 3))
    f = rng.normal(size=(n, 4)).astype(np.float32 if precision == "mixed" else np.float64)
    r48 = rng.integers(0, 1 << 48, size=n, dtype=np.uint64)
    return p, x, v, f, r48


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_round_trip(tmp_path, precision):
    p, x, v, f, r48 = _state(precision=precision)
    path = tmp_path / "ck.npz"
    lj.write_checkpoint(path, p, x, v, f, steps=123, forces_valid=True, deterministic=True, rng=r48)
    ck = lj.read_checkpoint(path)
    for name, _ in lj.lj_params._fields_:
        assert getattr(ck["params"], name) == getattr(p, name), name
    assert np.array_equal(ck["x"], x) and np.array_equal(ck["v"], v)
    assert ck["f"].dtype == f.dtype and np.array_equal(ck["f"], f)
    assert np.array_equal(ck["rng"], r48)
    assert ck["steps"] == 123 and ck["forces_valid"] and ck["deterministic"]


def test_without_rng_and_empty_system(tmp_path):
    p, x, v, f, _ = _state(n=0)
    path = tmp_path / "empty.npz"
    lj.write_checkpoint(path, p, x, v, f, forces_valid=False)
    ck = lj.read_checkpoint(path)
    assert ck["rng"] is None and ck["params"].n == 0 and not ck["forces_valid"] and ck["steps"] == 0


def test_int64_bit_patterns_are_accepted(tmp_path):
    p, x, v, f, r48 = _state()
    path = tmp_path / "ck.npz"
    lj.write_checkpoint(path, p, x, v, f, rng=r48.view(np.int64))
    assert np.array_equal(lj.read_checkpoint(path)["rng"], r48)


def test_bad_inputs_refused(tmp_path):
    p, x, v, f, r48 = _state()
    path = tmp_path / "ck.npz"
    with pytest.raises(ValueError):
        lj.write_checkpoint(path, p, x[:-1], v, f)
    with pytest.raises(ValueError):
        lj.write_checkpoint(path, p, x, v, f.astype(np.float64))    # mixed forces are float32
    bad = r48.copy()
    bad[3] = np.uint64(1 << 48)
    with pytest.raises(ValueError):
        lj.write_checkpoint(path, p, x, v, f, rng=bad)
    # a file of another format version, and one with a state array cut short
    lj.write_checkpoint(path, p, x, v, f, rng=r48)
    with np.load(path) as z:
        arrays = {k: z[k] for k in z.files}
    for key, value in (("version", np.int64(99)), ("x", x[:5])):
        other = dict(arrays)
        other[key] = value
        bad_path = tmp_path / f"bad_{key}.npz"
        np.savez(bad_path, **other)
        with pytest.raises(ValueError):
            lj.read_checkpoint(bad_path)
