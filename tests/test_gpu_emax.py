"""Derivative through the Thompson cut-off on the GPU: the boundary run
against the oracle's, the E_i derivative against common-random-number finite
differences, and the power gradient of the composition map with the ion
energy following the discharge voltage (Table S1 voltage lines)."""

import math

import numpy as np
import pytest

import workloads
from workloads import ELEMENTS
from workloads.measurement import calibration_points, measurement_patches, voltage_points

pytestmark = pytest.mark.gpu

QUAT = ("Ni", "Pd", "Pt", "Ru")


@pytest.fixture(scope="module")
def pkg():
    import paper_2411_14413_gb300 as p
    p.build()
    return p


def test_boundary_run_matches_the_oracle(pkg, oracle_mod):
    from paper_2411_14413_gb300 import _native as N

    sc = workloads.scene_single_ni(n=4000)
    tr = pkg.Transport(sc, records=True)
    tr.run(flags=N.SPUT_RUN_LAUNCH_AT_CUTOFF)
    g = tr.records()
    tr.close()
    o = oracle_mod.OracleScene(sc).run_all(at_cutoff=True)
    same = (g["prim"] == o["prim"]) & (g["cell"] == o["cell"])
    n = len(same)
    assert (~same).sum() <= 0.001 * n + 3 * math.sqrt(0.001 * n) + 1
    # atoms that land without a collision arrive with E_max
    direct = (g["ncoll"] == 0) & (g["prim"] >= 0)
    Em = oracle_mod.OracleScene(sc).emax(0)
    assert direct.sum() > 100 and np.allclose(g["E"][direct], Em, rtol=1e-5)


def test_ion_energy_gradient_matches_crn_finite_difference(pkg):
    from paper_2411_14413_gb300 import _native as N
    import torch

    sc = workloads.scene_quaternary(n_per_cathode=1_000_000)
    tr = pkg.Transport(sc, energy=False)
    cut = pkg.Transport(sc, energy=False)
    w = torch.zeros((4, 200, 200), dtype=torch.float64, device="cuda")
    w[:, 60:140, 60:140] = 1.0
    grad = torch.zeros(4, dtype=torch.float64, device="cuda")
    h = 20.0
    lr, fd = [], []
    for seed in range(4):
        tr.set_instances(sc)
        tr.run(seed=seed)
        cut.run(seed=seed, flags=N.SPUT_RUN_LAUNCH_AT_CUTOFF)
        N.check(N.load().sput_emax_backward(tr.h, w.data_ptr(), tr.t["counts"].data_ptr(), cut.t["counts"].data_ptr(),
                                            grad.data_ptr(), torch.cuda.current_stream().cuda_stream),
                "sput_emax_backward")
        torch.cuda.synchronize()
        lr.append(grad.cpu().numpy().copy())
        vals = []
        for sgn in (+1, -1):
            tr.set_instances(sc.with_ion_energy(400.0 + sgn * h))
            tr.run(seed=seed)
            vals.append((tr.t["counts"].double() * w).sum(dim=(1, 2)).cpu().numpy())
        fd.append((vals[0] - vals[1]) / (2 * h))
    tr.close()
    cut.close()
    lr, fd = np.array(lr), np.array(fd)
    for j in range(4):
        se = math.sqrt(lr[:, j].var(ddof=1) / 4 + fd[:, j].var(ddof=1) / 4)
        assert abs(lr[:, j].mean() - fd[:, j].mean()) < 5 * se + 0.05 * abs(fd[:, j].mean()), (j, lr[:, j], fd[:, j])


def test_power_gradient_with_voltage_coupling(pkg):
    """dL/dP_j of L = sum(g * composition) with E_i following the voltage line:
    the rate-line term plus the cut-off term, against central differences of
    the same seeded maps."""
    import torch
    from paper_2411_14413_gb300.adjoint import MapSetup

    patch, pts, ref = measurement_patches()
    sc = workloads.scene_quaternary(n_per_cathode=1_000_000)
    cal = []
    volt = []
    for s in QUAT:
        (p1, r1), (p2, r2) = calibration_points(s)
        cal.append([p1, r1, p2, r2, ELEMENTS[s].density, ELEMENTS[s].mass])
        (q1, v1), (q2, v2) = voltage_points(s)
        volt.append([q1, v1, q2, v2])
    ms = MapSetup(sc, patch, ref, np.array(cal), voltage=np.array(volt))
    power = np.array([20.0, 30.0, 12.0, 18.0])
    rng = np.random.default_rng(5)
    gcomp = torch.as_tensor(rng.normal(size=(len(pts), 4)), device="cuda")
    an, fd = [], []
    dP = 3.0
    for seed in range(3):
        ms.forward(0.5, power, seed)
        _, gp = ms.backward(gcomp, power)
        an.append(gp.cpu().numpy().copy())
        row = []
        for j in range(4):
            e = np.zeros(4)
            e[j] = dP
            lp = float((gcomp * ms.forward(0.5, power + e, seed)).sum())
            lm = float((gcomp * ms.forward(0.5, power - e, seed)).sum())
            row.append((lp - lm) / (2 * dP))
        fd.append(row)
    ms.close()
    an, fd = np.array(an), np.array(fd)
    for j in range(4):
        se = math.sqrt(an[:, j].var(ddof=1) / 3 + fd[:, j].var(ddof=1) / 3)
        assert abs(an[:, j].mean() - fd[:, j].mean()) < 5 * se + 0.1 * abs(fd[:, j].mean()), (j, an[:, j], fd[:, j])


def test_trajectory_parity_at_table_s1_ion_energies(pkg, oracle_mod):
    """Whole trajectories against the oracle with E_i from the Table S1 voltage
    lines at mid-range powers (DC near 300 V, the RF-driven Pd near 37 V, whose
    cut-off is only a few eV)."""
    sc = workloads.scene_quaternary(n_per_cathode=1500)
    power = {"Ni": 20.0, "Pd": 30.0, "Pt": 12.0, "Ru": 18.0}
    Ei = []
    for s in QUAT:
        (q1, v1), (q2, v2) = voltage_points(s)
        Ei.append(v1 + (v2 - v1) * (power[s] - q1) / (q2 - q1))
    sc = sc.with_ion_energy(Ei)
    tr = pkg.Transport(sc, records=True)
    tr.run()
    g = tr.records()
    tr.close()
    o = oracle_mod.OracleScene(sc)
    assert o.emax(1) < 10.0   # the RF-driven Pd launches below 10 eV
    r = o.run_all()
    same = (g["prim"] == r["prim"]) & (g["cell"] == r["cell"])
    n = len(same)
    assert (~same).sum() <= 0.001 * n + 3 * math.sqrt(0.001 * n) + 1, (~same).sum()
