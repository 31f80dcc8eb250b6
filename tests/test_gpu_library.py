"""Tilt scan on the GPU: the maps of all tilts from one launch (checked against
the oracle's composition arithmetic on the same counts), and the recovery of
the tilt of a map simulated at a tilt between the scanned ones, by the
compositional-area criterion and by least squares with a fitted reference."""

import numpy as np
import pytest

import workloads
from workloads import ELEMENTS
from workloads.measurement import calibration_points, measurement_patches

pytestmark = pytest.mark.gpu

EL = ("Pd", "Pt", "Ru")


@pytest.fixture(scope="module")
def pkg():
    import paper_2411_14413_gb300 as p
    p.build()
    return p


def _calibration():
    cal = []
    for s in EL:
        (p1, r1), (p2, r2) = calibration_points(s)
        cal.append([p1, r1, p2, r2, ELEMENTS[s].density, ELEMENTS[s].mass])
    return np.array(cal)


def test_tilt_scan_maps_and_diagnosis(pkg, oracle_mod):
    from paper_2411_14413_gb300 import library

    cal, power = _calibration(), np.array([30.0, 12.0, 18.0])
    patch, pts, ref = measurement_patches()
    # 1e8 atoms per cathode, as in the paper: the count noise of the reference
    # patch moves a whole map, so fewer atoms blur the tilt estimate
    true_tilt, n = 30.6, 100_000_000
    meas_sc = workloads.scene_tilt_scan([true_tilt], elements=EL, n_per_cathode=n, seed=123)
    tr = pkg.Transport(meas_sc, energy=False, prim_counts=False)
    meas = library.composition_maps(tr, 3, patch, ref, cal, power, seed=123)[0].cpu().numpy()
    tr.close()
    tilts = np.arange(27.0, 34.01, 1.0)
    sc = workloads.scene_tilt_scan(tilts, elements=EL, n_per_cathode=n)
    tr = pkg.Transport(sc, energy=False, prim_counts=False)
    sims = library.composition_maps(tr, 3, patch, ref, cal, power, seed=0).cpu().numpy()
    counts = tr.t["counts"].cpu().numpy().reshape(len(tilts), 3, -1).astype(np.float64)
    tr.close()
    rates = np.array([oracle_mod.rate_line(calibration_points(s), P)[0] for s, P in zip(EL, power)])
    for t in (0, 4, 7):
        want, _ = oracle_mod.composition(counts[t], patch, ref, rates, cal[:, 4], cal[:, 5])
        assert np.allclose(sims[t], want, rtol=1e-12, atol=1e-10)
    d = library.diagnose_tilt(meas, tilts, sims)
    print("tilt diagnosis:", {k: d[k] for k in ("tilt_area", "tilt_lsq", "area_measured")},
          "areas", np.round(d["areas"], 5), "mse", np.round(d["mse"], 4))
    # a larger common tilt shrinks the covered compositional area, step by step
    assert all(a > b for a, b in zip(d["areas"], d["areas"][1:])), d["areas"]
    assert d["tilt_area"] is not None and abs(d["tilt_area"] - true_tilt) < 0.5, d
    # point-by-point least squares with a fitted reference: per-element factors absorb
    # the count noise of the reference patch that every map is normalised to
    assert abs(d["tilt_lsq"] - true_tilt) < 0.5, d
    assert np.all(np.abs(np.asarray(d["lsq_factors"]) - 1.0) < 0.05), d["lsq_factors"]
