"""Pins for the oracle's composition conversion and the calibration data."""

import numpy as np

from workloads import ELEMENTS
from workloads.measurement import TABLE_S1, calibration_points, measurement_patches


def test_table_s1_rates_are_thickness_over_time():
    """Every printed rate of Table S1 equals average thickness / deposition time
    within the rounding of the printed thickness (0.05 nm) and rate (half a
    unit of its last digit); this fixes the garbled "27 60" as 2760 s (a tenfold
    other reading would miss by a factor of 10)."""
    for el, supplies in TABLE_S1.items():
        for rows in supplies.values():
            for (_p, t, thick, printed) in rows:
                last = 10 ** (np.floor(np.log10(printed)) - 3)   # four significant digits
                tol = 0.05 / thick * printed + 0.5 * last
                assert abs(thick / t - printed) <= tol, (el, printed, thick / t)


def test_measurement_grid_has_342_points():
    patch, pts, ref = measurement_patches()
    assert len(pts) == 342 and patch.max() == 341
    assert np.all(np.hypot(pts[:, 0], pts[:, 1]) <= 45.0)
    assert np.allclose(pts[ref], 0.0)
    assert np.all(np.bincount(patch[patch >= 0]) == 64)   # 4 mm patch = 8 x 8 cells of 0.5 mm


def test_composition_special_cases(oracle_mod):
    patch, pts, ref = measurement_patches()
    n_cells = patch.size
    rng = np.random.default_rng(0)
    base = rng.integers(50, 200, size=n_cells).astype(float)
    counts = np.stack([base] * 4)
    ones = np.ones(4)
    # identical elements (same rate, density, mass) -> 25 at.% everywhere
    comp, _ = oracle_mod.composition(counts, patch, ref, ones, ones, ones)
    assert np.allclose(comp, 25.0)
    # one element absent -> the others share 100 %, the absent one 0
    c2 = counts.copy()
    c2[3][:] = 0.0
    c2[3][patch == ref] = 1.0   # keep the reference finite
    comp, _ = oracle_mod.composition(c2, patch, ref, ones, ones, ones)
    off = np.arange(len(pts)) != ref
    assert np.allclose(comp[off, 3], 0.0) and np.allclose(comp[off, :3].sum(1), 100.0)
    # at the reference point the at.% ratio is rate*density/mass ratio
    dens = np.array([ELEMENTS[s].density for s in ("Ni", "Pd", "Pt", "Ru")])
    mass = np.array([ELEMENTS[s].mass for s in ("Ni", "Pd", "Pt", "Ru")])
    rates = np.array([oracle_mod.rate_line(calibration_points(s), 20.0)[0] for s in ("Ni", "Pd", "Pt", "Ru")])
    comp, _ = oracle_mod.composition(counts, patch, ref, rates, dens, mass)
    w = rates * dens / mass
    assert np.allclose(comp[ref], 100 * w / w.sum())


def test_rate_line_through_calibration_points(oracle_mod):
    for s in ("Ni", "Pd", "Pt", "Ru"):
        pts = calibration_points(s)
        for p, r in pts:
            assert abs(oracle_mod.rate_line(pts, p)[0] - r) < 1e-15
