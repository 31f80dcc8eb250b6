"""Sharded runs on one GPU: the ranks' ticket ranges, transported one after
another into the same tallies, give the single-run tallies bit-exactly (the
integer sum a multi-GPU job performs once per run)."""

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2411_14413_gb300 as p
    p.build()
    return p


@pytest.mark.parametrize("world", [2, 3])
def test_run_shard_accumulates_to_the_full_run(pkg, world):
    sc = workloads.scene_quaternary(n_per_cathode=50_000)
    full = pkg.Transport(sc, energy=True)
    st = full.run(seed=7)
    parts = pkg.Transport(sc, energy=True)
    n = 0
    for r in range(world):
        s = pkg.shard.run_shard(parts, r, world, seed=7, accumulate=r > 0)
        n += s.particles
    assert n == st.particles == sc.total_particles
    for k in ("counts", "prim_counts", "timed_out"):
        assert np.array_equal(full.t[k].cpu().numpy(), parts.t[k].cpu().numpy()), k
    assert np.allclose(full.t["energy"].cpu().numpy(), parts.t["energy"].cpu().numpy(), rtol=1e-12, atol=1e-9)
    full.close()
    parts.close()
