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
