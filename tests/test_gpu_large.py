"""The large shielded chamber at 3 Pa (64 primitives, 512 x 512 grid, arrival
energy and angle histograms): per-particle parity with the oracle on a
sample, histogram consistency, and conservation at a larger count."""

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


def test_large_scene_parity_and_histograms(torch, pkg, oracle_mod):
    sc = workloads.scene_large_shielded(n=800)
    assert len(sc.prims) == 64
    tr = pkg.Transport(sc, records=True, energy=True)
    st = tr.run()
    g = tr.records()
    tal = {k: v.cpu().numpy() for k, v in tr.t.items() if k != "records"}
    tr.close()
    assert st.particles == 800
    o = oracle_mod.OracleScene(sc).run_all()
    same = (g["prim"] == o["prim"]) & (g["cell"] == o["cell"])
    n = len(same)
    # 3 Pa: hundreds of collisions per atom, so decision flips accumulate; the
    # 99.9 % budget is kept for particles with fewer than 200 collisions and
    # 99 % for all
    short = o["ncoll"] < 200
    bad_short = int((~same[short]).sum())
    assert bad_short <= 0.001 * short.sum() + 3 * math.sqrt(0.001 * short.sum()) + 1, bad_short
    assert same.mean() > 0.99, same.mean()
    # GPU histograms are the binned GPU records; the oracle's binned outcomes agree
    # except for the particles that differ
    t_or = oracle_mod.tally(sc, o)
    t_gp = oracle_mod.tally(sc, {**g, "inst": np.zeros(n, np.int64), "cos": g["cos"]})
    assert np.array_equal(tal["hist_E"], t_gp["hist_E"])
    assert np.array_equal(tal["hist_A"], t_gp["hist_A"])
    diff_E = np.abs(tal["hist_E"] - t_or["hist_E"]).sum()
    assert diff_E <= 2 * (~same).sum() + 4
    assert int(tal["counts"].sum()) == int(tal["hist_E"].sum()) == int(tal["hist_A"].sum())


def test_large_scene_conservation(torch, pkg):
    sc = workloads.scene_large_shielded(n=2_000_000)
    tr = pkg.Transport(sc, energy=True)
    st = tr.run(seed=4)
    assert st.particles == 2_000_000 and st.device_status == 0
    assert int(tr.t["prim_counts"].sum() + tr.t["timed_out"].sum()) == 2_000_000
    assert st.collisions / st.particles > 50      # 3 Pa: many collisions per atom
    tr.close()
