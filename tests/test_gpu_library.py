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


TRUE_TILT, N_PER_CATHODE = 30.6, 100_000_000
POWER = np.array([30.0, 12.0, 18.0])


@pytest.fixture(scope="module")
def measured(pkg):
    """The 'measured' map: the library simulated at 30.6 degrees with its own seed.
    1e8 atoms per cathode, as in the paper: the count noise of the reference patch
    moves a whole map, so fewer atoms blur the tilt estimate."""
    from paper_2411_14413_gb300 import library

    patch, pts, ref = measurement_patches()
    meas_sc = workloads.scene_tilt_scan([TRUE_TILT], elements=EL, n_per_cathode=N_PER_CATHODE, seed=123)
    tr = pkg.Transport(meas_sc, energy=False, prim_counts=False)
    meas = library.composition_maps(tr, 3, patch, ref, _calibration(), POWER, seed=123)[0].cpu().numpy()
    tr.close()
    return meas


def test_tilt_scan_maps_and_diagnosis(pkg, oracle_mod, measured):
    from paper_2411_14413_gb300 import library

    cal, power = _calibration(), POWER
    patch, pts, ref = measurement_patches()
    true_tilt, n, meas = TRUE_TILT, N_PER_CATHODE, measured
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


def test_tilt_newton_through_the_composition_adjoint(pkg, measured):
    """Newton steps on the tilt from the nominal 30 degrees: each step is one batched launch
    of the library at (t - h, t, t + h) with common random numbers across the three tilts;
    the slope is the composition adjoint's dL/dcounts contracted with the central count
    difference.  The 30.6-degree map is recovered within 0.5 degrees.  The three tilts
    share one realisation of the simulation's count noise, which no averaging over tilts
    reduces (the scan's quadratic averages over eight independent maps), so the Newton
    simulation runs 4e8 atoms per cathode."""
    from paper_2411_14413_gb300 import library

    patch, pts, ref = measurement_patches()

    def make_scene(tilts):
        return workloads.scene_tilt_scan(tilts, elements=EL, n_per_cathode=4 * N_PER_CATHODE,
                                         common_random_numbers=True)

    adj = library.TiltAdjoint(make_scene, measured, patch, ref, _calibration(), POWER, seed=0)
    t, hist = library.fit_tilt_newton(adj.evaluate, 30.0, h=1.0, iters=6, tol=0.05)
    print("tilt newton:", round(t, 3), [(round(r["t"], 3), round(r["slope"], 5), round(r["curv"], 5),
                                        round(r["step"], 3)) for r in hist])
    assert abs(t - TRUE_TILT) < 0.5, hist
    # the adjoint slope and the difference of the fitted losses agree in sign and roughly in size
    r = hist[0]
    fd = (r["losses"][2] - r["losses"][0]) / 2.0
    assert r["slope"] * fd > 0 and abs(r["slope"] - fd) < 0.5 * abs(fd) + 1e-4, r
