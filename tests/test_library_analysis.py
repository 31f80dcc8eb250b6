"""Host-side library analysis: the compositional area against closed forms
and a brute-force hull, and the tilt estimate on maps with a known answer."""

import itertools
import math

import numpy as np
import pytest

from paper_2411_14413_gb300 import library


def _gift_wrap_area(p):
    """Area of the convex hull of 2-D points by gift wrapping + shoelace."""
    p = np.asarray(p, float)
    start = int(np.lexsort((p[:, 1], p[:, 0]))[0])
    hull, cur = [], start
    while True:
        hull.append(cur)
        nxt = (cur + 1) % len(p)
        for j in range(len(p)):
            a, b = p[nxt] - p[cur], p[j] - p[cur]
            cross = a[0] * b[1] - a[1] * b[0]
            if cross < 0 or (cross == 0 and np.dot(b, b) > np.dot(a, a)):
                nxt = j
        cur = nxt
        if cur == start:
            break
    h = p[hull]
    return 0.5 * abs(np.dot(h[:, 0], np.roll(h[:, 1], -1)) - np.dot(h[:, 1], np.roll(h[:, 0], -1)))


def test_area_of_the_whole_simplex_is_one():
    assert library.compositional_area(np.array([[100, 0, 0], [0, 100, 0], [0, 0, 100], [30, 30, 40]])) == pytest.approx(1.0)
    assert library.compositional_area(100 * np.eye(4)) == pytest.approx(1.0)


def test_area_of_sub_simplices_closed_form():
    # the triangle of compositions with every element >= a (at.%) is a simplex scaled by (1 - 3a/100)
    for a in (5.0, 20.0):
        pts = np.array([[100 - 2 * a, a, a], [a, 100 - 2 * a, a], [a, a, 100 - 2 * a]])
        assert library.compositional_area(pts) == pytest.approx((1 - 3 * a / 100) ** 2)
        pts4 = np.full((4, 4), a) + np.eye(4) * (100 - 4 * a)
        assert library.compositional_area(pts4) == pytest.approx((1 - 4 * a / 100) ** 3)


def test_area_matches_brute_force_hull_on_random_maps():
    rng = np.random.default_rng(2)
    for _ in range(5):
        x = rng.dirichlet([4, 3, 2], size=60) * 100
        # the simplex share is the hull area in the (x1, x2) fractions times 2! = 2
        want = 2 * _gift_wrap_area(x[:, :2] / 100)
        assert library.compositional_area(x) == pytest.approx(want, rel=1e-12)


def test_diagnose_tilt_recovers_a_known_shrink():
    """Maps whose spread around the centre shrinks linearly with tilt: the area
    criterion and the least-squares criterion both return the true tilt."""
    rng = np.random.default_rng(0)
    base = rng.dirichlet([5, 5, 5], size=200) * 100 - 100 / 3

    def lib(t):
        return 100 / 3 + base * (1.0 - 0.02 * (t - 30.0))

    tilts = np.arange(26.0, 34.01, 1.0)
    d = library.diagnose_tilt(lib(30.6), tilts, [lib(t) for t in tilts])
    assert d["tilt_area"] == pytest.approx(30.6, abs=0.05)
    assert d["tilt_lsq"] == pytest.approx(30.6, abs=1e-3)   # per-map factors fitted numerically
    assert all(a > b for a, b in zip(d["areas"], d["areas"][1:]))


def test_fit_tilt_absorbs_reference_patch_scale():
    """A measured map whose elements are rescaled (the effect of a noisy count in the
    reference patch every map is normalised to): the least-squares fit with free
    per-element factors returns the true tilt and the factors.  The tilt dependence
    is a smooth rotation of the points around the centre, linear within a scan step."""
    rng = np.random.default_rng(4)
    base = rng.dirichlet([6, 6, 6], size=300) * 100 - 100 / 3

    def lib(t):
        a = math.radians(4.0 * (t - 30.0))
        # rotate within the plane of compositions (rows keep summing to 100)
        u = np.array([1.0, -1.0, 0.0]) / math.sqrt(2)
        v = np.array([1.0, 1.0, -2.0]) / math.sqrt(6)
        x, y = base @ u, base @ v
        xr, yr = x * math.cos(a) - y * math.sin(a), x * math.sin(a) + y * math.cos(a)
        return 100 / 3 + np.outer(xr, u) + np.outer(yr, v)

    tilts = np.arange(28.0, 33.01, 0.5)
    k_true = np.array([1.0, 1.006, 0.993])
    meas = library._rescale(lib(30.5), np.log(k_true))
    # every simulated map with its own reference error: the per-map factors absorb them
    rng = np.random.default_rng(9)
    sims = [library._rescale(lib(x), rng.normal(0.0, 0.005, 3)) for x in tilts]
    t, k, mse = library.fit_tilt(meas, tilts, sims)
    assert t == pytest.approx(30.5, abs=0.02)
    assert np.min(mse) < 1e-3
    d = library.diagnose_tilt(meas, tilts, sims)
    assert d["tilt_lsq"] == pytest.approx(30.5, abs=0.02)
    # a single map's factors recover the measured map's reference error exactly
    k1, m1 = library.fit_reference(lib(30.5), meas)
    assert np.allclose(k1, k_true, rtol=1e-6) and m1 < 1e-12


def test_fitted_loss_grad_matches_finite_differences():
    """The gradient of the fitted-reference loss (the minimum over the per-element
    factors) equals its central differences in single map entries: at the optimal
    factors the loss is stationary in them, so the partial derivative at fixed
    factors is the whole derivative."""
    rng = np.random.default_rng(11)
    sim = rng.dirichlet([4, 4, 4], size=40) * 100
    meas = library._rescale(rng.dirichlet([4, 4, 4], size=40) * 100, [0.0, 0.02, -0.01])
    loss, k, grad = library.fitted_loss_grad(sim, meas)
    assert loss == pytest.approx(library.fit_reference(sim, meas)[1], rel=1e-12)
    assert grad.shape == sim.shape
    eps = 1e-4
    for i, j in [(0, 0), (3, 1), (17, 2), (39, 0), (25, 1)]:
        sp, sm = sim.copy(), sim.copy()
        sp[i, j] += eps
        sm[i, j] -= eps
        fd = (library.fit_reference(sp, meas)[1] - library.fit_reference(sm, meas)[1]) / (2 * eps)
        assert grad[i, j] == pytest.approx(fd, rel=1e-4, abs=1e-9)
    # a map against itself: zero loss, unit factors, zero gradient
    l0, k0, g0 = library.fitted_loss_grad(sim, sim)
    assert l0 < 1e-20 and np.allclose(k0, 1.0, atol=1e-8) and np.allclose(g0, 0.0, atol=1e-8)


def test_fit_tilt_newton_recovers_a_rotation_tilt():
    """Newton steps on the fitted-reference loss, with the slope from the loss gradient in
    the map contracted with the central difference of the maps in tilt (the contraction
    the GPU path makes through the composition adjoint on counts), reach the true tilt of a
    measured map with a reference error from a start 1.5 degrees away."""
    rng = np.random.default_rng(4)
    base = rng.dirichlet([6, 6, 6], size=300) * 100 - 100 / 3
    u = np.array([1.0, -1.0, 0.0]) / math.sqrt(2)
    v = np.array([1.0, 1.0, -2.0]) / math.sqrt(6)

    def lib(t):
        a = math.radians(4.0 * (t - 30.0))
        x, y = base @ u, base @ v
        xr, yr = x * math.cos(a) - y * math.sin(a), x * math.sin(a) + y * math.cos(a)
        return 100 / 3 + np.outer(xr, u) + np.outer(yr, v)

    meas = library._rescale(lib(30.5), np.log([1.0, 1.006, 0.993]))

    def evaluate(t, h):
        lm = library.fit_reference(lib(t - h), meas)[1]
        lp = library.fit_reference(lib(t + h), meas)[1]
        loss, k, g = library.fitted_loss_grad(lib(t), meas)
        slope = float((g * (lib(t + h) - lib(t - h)) / (2 * h)).sum())
        return {"t": t, "loss": loss, "slope": slope, "curv": (lp - 2 * loss + lm) / h ** 2}

    t, hist = library.fit_tilt_newton(evaluate, 29.0, h=1.0)
    assert t == pytest.approx(30.5, abs=0.01)
    assert len(hist) <= 6 and abs(hist[-1]["step"]) < 0.02
    # the slope agrees with the difference of the losses and points downhill from the start
    r = evaluate(29.0, 1e-3)
    lm = library.fit_reference(lib(29.0 - 1e-3), meas)[1]
    lp = library.fit_reference(lib(29.0 + 1e-3), meas)[1]
    assert r["slope"] == pytest.approx((lp - lm) / 2e-3, rel=1e-3)
    assert r["slope"] < 0


def test_fit_tilt_newton_brackets_a_jagged_slope():
    """A loss whose slope carries a jagged term of +-0.25 in alternate 0.1-degree bands (the
    finite-sample slope near the minimum): from 29 degrees the bare Newton step cycles
    between about 30.375 and 30.625 for ever; the bracket ends the iteration inside the
    sign change, near the true minimum."""

    def evaluate(t, h):
        jag = 0.25 * (1.0 if int(math.floor(t / 0.1)) % 2 == 0 else -1.0)
        return {"t": t, "loss": (t - 30.5) ** 2, "slope": 2.0 * (t - 30.5) + jag, "curv": 2.0}

    # the bare Newton iteration cycles
    t, seen = 29.0, []
    for _ in range(12):
        t += float(np.clip(-evaluate(t, 1.0)["slope"] / 2.0, -1.0, 1.0))
        seen.append(round(t, 3))
    assert len(set(seen[-6:])) == 2
    t, hist = library.fit_tilt_newton(evaluate, 29.0, h=1.0, iters=20, tol=0.02)
    assert abs(t - 30.5) < 0.15
    assert len(hist) < 20 and hist[-1]["step"] != 0.0
