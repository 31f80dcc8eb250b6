"""Temperature score d ln p(path)/dT (pressure fixed) on the GPU: the
stationary-gas identity, the per-cell sums against the oracle's per-particle
scores, and common-random-number finite differences in T."""

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


def test_stationary_gas_identity(pkg):
    """Gas at rest: T acts only through n_g = p/(k_B T), so score_T = -score/T.
    (Hard spheres: with the Moliere cross section, which grows without bound as
    the atom slows down, atoms in a gas at rest never stop colliding.)"""
    sc = workloads.scene_single_ni(n=20_000, physics={"interaction": "hard_sphere", "gas_motion": "stationary",
                                                      "max_collisions": 150})
    tr = pkg.Transport(sc, score=True, score_T=True)
    tr.run()
    s, sT = tr.t["score"].cpu().numpy(), tr.t["score_T"].cpu().numpy()
    tr.close()
    scale = np.abs(s).max() / sc.T
    assert scale > 0
    assert np.max(np.abs(sT + s / sc.T)) < 1e-5 * scale


def test_score_T_tally_matches_the_oracle(pkg, oracle_mod):
    sc = workloads.scene_single_ni(n=3000)
    tr = pkg.Transport(sc, score_T=True, records=True)
    tr.run()
    g = tr.records()
    got = tr.t["score_T"].cpu().numpy().ravel()
    tr.close()
    o = oracle_mod.OracleScene(sc).run_all(score_T=True)
    same = (g["prim"] == o["prim"]) & (g["cell"] == o["cell"]) & (g["ncoll"] == o["ncoll"])
    assert same.mean() > 0.999
    on = (o["cell"] >= 0) & same
    want = np.bincount(o["cell"][on], weights=o["score_T"][on], minlength=got.size)
    # cells holding a particle that landed differently are left out
    bad = np.unique(np.concatenate([g["cell"][~same], o["cell"][~same]]))
    keep = np.ones(got.size, bool)
    keep[bad[bad >= 0]] = False
    tol = 2e-4 * np.abs(o["score_T"]).max() + 1e-4 * np.abs(want)
    assert np.all(np.abs(got[keep] - want[keep]) <= tol[keep])


def test_temperature_gradient_matches_crn_finite_difference(pkg):
    """d/dT of the arrivals in a central region: LR (sum of w * score_T) against
    central finite differences at T (1 +- h) with common random numbers."""
    from paper_2411_14413_gb300 import _native as N
    import torch

    base = workloads.scene_quaternary(n_per_cathode=1_000_000)
    h = 0.03
    tr = pkg.Transport(base, score_T=True)
    sides = []
    for sgn in (+1, -1):
        sc = workloads.scene_quaternary(n_per_cathode=1_000_000, T=base.T * (1 + sgn * h))
        sides.append(pkg.Transport(sc, energy=False))
    w = torch.zeros((4, 200, 200), dtype=torch.float64, device="cuda")
    w[:, 60:140, 60:140] = 1.0
    grad = torch.zeros(4, dtype=torch.float64, device="cuda")
    lr, fd = [], []
    for seed in range(4):
        tr.run(seed=seed)
        N.check(N.load().sput_backward(tr.h, w.data_ptr(), tr.t["score_T"].data_ptr(), grad.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream), "sput_backward")
        torch.cuda.synchronize()
        lr.append(grad.cpu().numpy().copy())
        vals = []
        for t in sides:
            t.run(seed=seed)
            vals.append((t.t["counts"].double() * w).sum(dim=(1, 2)).cpu().numpy())
        fd.append((vals[0] - vals[1]) / (2 * h * base.T))
    for t in [tr] + sides:
        t.close()
    lr, fd = np.array(lr), np.array(fd)
    for j in range(4):
        se = math.sqrt(lr[:, j].var(ddof=1) / 4 + fd[:, j].var(ddof=1) / 4)
        assert abs(lr[:, j].mean() - fd[:, j].mean()) < 5 * se + 0.05 * abs(fd[:, j].mean()), (j, lr[:, j], fd[:, j])


def test_trajectory_parity_at_another_gas_temperature(pkg, oracle_mod):
    """Whole trajectories against the oracle with the gas at 500 K (rate and
    rejection tables built for another Maxwellian spread)."""
    sc = workloads.scene_single_ni(n=5000, T=500.0)
    tr = pkg.Transport(sc, records=True)
    tr.run()
    g = tr.records()
    tr.close()
    o = oracle_mod.OracleScene(sc).run_all()
    same = (g["prim"] == o["prim"]) & (g["cell"] == o["cell"])
    n = len(same)
    assert (~same).sum() <= 0.001 * n + 3 * math.sqrt(0.001 * n) + 1, (~same).sum()
