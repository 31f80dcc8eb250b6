"""Diffusion shortcut for thermalised atoms on the GPU: per-particle parity
with the oracle's shortcut, and the approximation against the full Monte
Carlo at 3 Pa."""

import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2411_14413_gb300 as p
    p.build()
    return p


def test_shortcut_parity_with_the_oracle(pkg, oracle_mod):
    sc = workloads.scene_single_ni(n=3000, pressure=3.0, physics={"thermal_switch_eV": 0.1})
    tr = pkg.Transport(sc, records=True)
    st = tr.run()
    g = tr.records()
    tr.close()
    o = oracle_mod.OracleScene(sc).run_all()
    same = (g["prim"] == o["prim"]) & (g["cell"] == o["cell"])
    n = len(same)
    assert st.particles == n and o["ncoll"].mean() > 20
    assert (~same).sum() <= 0.001 * n + 3 * math.sqrt(0.001 * n) + 1, (~same).sum()


def test_shortcut_rejects_what_it_does_not_define(pkg):
    from paper_2411_14413_gb300 import _native as N

    sc = workloads.scene_single_ni(n=100, physics={"thermal_switch_eV": 0.1})
    tr = pkg.Transport(sc, score_T=True)
    with pytest.raises(N.SputError):
        tr.run()
    tr.close()


def test_shortcut_against_full_monte_carlo_at_3_pa(pkg):
    """Large shielded chamber at 3 Pa (hundreds of collisions per atom): with the
    switch at 0.1 eV (about 2.6 x 3/2 kT) the landing fractions on every primitive
    and the substrate profile on an 8 x 8 coarse grid agree with the exact model
    to statistical noise, several times faster."""
    res = {}
    for esw in (0.0, 0.1):
        sc = workloads.scene_large_shielded(n=4_000_000, physics={"thermal_switch_eV": esw})
        tr = pkg.Transport(sc, energy=False)
        tr.run(seed=9)
        st = tr.run(seed=1)
        c = tr.t["counts"].cpu().numpy().astype(float)[0]
        pc = tr.t["prim_counts"].cpu().numpy()[0] / st.particles
        tr.close()
        ny, nx = c.shape
        coarse = np.zeros((8, 8))
        np.add.at(coarse, (((np.arange(ny) * 8) // ny)[:, None], ((np.arange(nx) * 8) // nx)[None, :]), c)
        res[esw] = (st.kernel_ms, c.sum() / st.particles, pc, coarse)
    full, fast = res[0.0], res[0.1]
    print("shortcut: speedup %.2f, substrate %.5f vs %.5f" % (full[0] / fast[0], fast[1], full[1]))
    assert full[0] / fast[0] > 3.0
    assert abs(fast[1] / full[1] - 1) < 0.015
    assert np.max(np.abs(fast[2] - full[2])) < 0.01
    z = (fast[3] - full[3]) / np.sqrt(fast[3] + full[3] + 1)
    assert np.sqrt((z ** 2).mean()) < 1.6 and np.abs(z).max() < 4.5
