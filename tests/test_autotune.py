"""Autotuner: cache keys and round trip (CPU); on a GPU, the tuned settings
give the same forces as the defaults and a second call hits the cache."""
import numpy as np
import pytest

from paper_0709_3225_gb300 import inputs


def test_bucket_key_and_cache_round_trip(tmp_path):
    from paper_0709_3225_gb300 import autotune
    k1 = autotune.bucket_key("system-mixed", 4_000_000, 0.8442, gpu="GB300")
    k2 = autotune.bucket_key("system-mixed", 3_900_000, 0.86, gpu="GB300")
    k3 = autotune.bucket_key("system-mixed", 131_072, 0.8442, gpu="GB300")
    assert k1 == k2 and k1 != k3
    assert k1 == "GB300|system-mixed|N2^22|rho0.85"
    path = str(tmp_path / "cache.json")
    autotune.store_cache(k1, {"kernel": 0, "gw": 16}, path)
    autotune.store_cache(k3, {"kernel": 1, "gw": 0}, path)
    data = autotune.load_cache(path)
    assert data[k1] == {"kernel": 0, "gw": 16} and data[k3]["kernel"] == 1
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}


@pytest.mark.gpu
def test_tune_system_and_batch(tmp_path):
    import torch
    from paper_0709_3225_gb300 import autotune, lj
    path = str(tmp_path / "tune.json")
    x, L = inputs.jittered_fcc(12, 0.8442, 0.1, 3)
    s = lj.System(x, inputs.velocities(x.shape[0], 1.0, 3), L)
    s.forces()
    ref = s.f.clone()
    x_before = s.x.clone()
    r = autotune.tune_system(s, 0.8442, steps=4, warmup=3, path=path)
    assert not any("error" in t for t in r["trials"]), r["trials"]
    assert not r["cached"] and len(r["trials"]) == len(autotune.system_candidates("mixed"))
    assert {t["subdiv"] for t in r["trials"]} == {1, 2}
    assert torch.equal(s.x, x_before)                 # tuning works on a copy
    s.forces()
    assert float((s.f[:, :3] - ref[:, :3]).abs().max()) <= 1e-4 * float(ref[:, :3].abs().max())
    r2 = autotune.tune_system(s, 0.8442, path=path)
    assert r2["cached"] and r2["kernel"] == r["kernel"]
    s.close()
    e = inputs.ensemble(4, seed=3, n_lo=500, n_hi=3000)
    xs, vs = inputs.ensemble_state(e)
    b = lj.Batch(xs, vs, e.box)
    b.forces()
    bref = b.f.clone()
    rb = autotune.tune_batch(b, float(np.mean(e.rho)), steps=3, warmup=3, path=path)
    assert not rb["cached"]
    assert {t["subdiv"] for t in rb["trials"]} == {1, 2}    # the cell size is a tuning dimension
    b.forces()
    rms = float(bref[:, :3].double().pow(2).sum(dim=1).mean().sqrt())
    assert bool(((b.f[:, :3] - bref[:, :3]).double().abs() <= 1e-5 * (bref[:, :3].double().abs() + rms)).all())
    assert autotune.tune_batch(b, float(np.mean(e.rho)), path=path)["cached"] == (rb["subdiv"] == 1)
    b.check()
    b2 = autotune.batch_for(b, dict(rb, subdiv=2))     # the batch rebuilt with half-size cells
    assert b2.cell_subdiv == 2
    b2.forces()
    assert bool(((b2.f[:, :3] - bref[:, :3]).double().abs() <= 1e-5 * (bref[:, :3].double().abs() + rms)).all())
    b2.check()
    b2.close()
