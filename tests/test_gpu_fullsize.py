"""Parity at the sizes bench.py times, in its launch configuration, on sampled particles the
oracle recomputes one by one.

* The 512-instance sweep (4 cathodes x 16 pressures x 8 tilts) at one tenth of its particle
  counts (2.7e8 atoms), autotuned as the bench does.
* The large shielded chamber at 3 Pa with 1e8 atoms (568 collisions per atom), the surface test
  by cell masks.

Both: at least 99.9 % of the sampled particles land in the oracle's cell (three binomial
standard deviations of that budget allowed), and every atom is accounted for."""

import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def pkg():
    import paper_2411_14413_gb300 as p
    p.build()
    return p


def _check_sampled(tr, sc, oracle_mod, n_sample, seed):
    rec = tr.t["records"]
    prefix = np.concatenate([[0], np.cumsum([int(i["n"]) for i in sc.instances])])
    rng = np.random.default_rng(seed)
    tick = np.sort(rng.choice(prefix[-1], n_sample, replace=False))
    import torch as t
    r = rec[t.from_numpy(tick).to(rec.device)].cpu().numpy()
    inst = np.searchsorted(prefix, tick, side="right") - 1
    o = oracle_mod.OracleScene(sc).run_ids(inst.astype(np.int32), (tick - prefix[inst]).astype(np.uint64))
    same = (r[:, 0] == o["prim"]) & (r[:, 1] == o["cell"])
    allowed = 0.001 * n_sample + 3 * math.sqrt(0.001 * n_sample) + 1
    return int((~same).sum()), allowed, o


def test_sweep_at_bench_size(torch, pkg, oracle_mod):
    sc = workloads.scene_tilt_pressure_sweep()
    sc = sc.with_particles([max(1, int(i["n"] * 0.1)) for i in sc.instances])
    N = sc.total_particles
    assert N > 2.5e8
    tr = pkg.Transport(sc, records=True, energy=False)
    tr.autotune(sample_tickets=20_000_000)
    st = tr.run(seed=sc.seed)
    assert st.particles == N and st.device_status == 0
    assert int(tr.t["prim_counts"].sum() + tr.t["timed_out"].sum()) == N
    bad, allowed, o = _check_sampled(tr, sc, oracle_mod, 3000, 11)
    tr.close()
    assert bad <= allowed, (bad, allowed)


def test_large_scene_at_bench_size(torch, pkg, oracle_mod):
    sc = workloads.scene_large_shielded(n=100_000_000)
    tr = pkg.Transport(sc, records=True, energy=True)
    st = tr.run(seed=sc.seed)
    assert st.particles == 100_000_000 and st.device_status == 0
    assert int(tr.t["prim_counts"].sum() + tr.t["timed_out"].sum()) == 100_000_000
    assert int(tr.t["hist_E"].sum()) == int(tr.t["counts"].sum()) == int(tr.t["hist_A"].sum())
    assert st.collisions / st.particles > 500
    bad, allowed, o = _check_sampled(tr, sc, oracle_mod, 1500, 12)
    tr.close()
    assert bad <= allowed, (bad, allowed)
    assert np.median(o["ncoll"]) > 100
