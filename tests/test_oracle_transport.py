"""Pins for the oracle's flights, surface test and tallies: brute-force ray
marching, exponential survival (Eq. for lambda with constant lambda_m), the
vacuum cosine-law deposition profile, and integer conservation."""

import copy
import math

import numpy as np
import pytest
from scipy import special, stats

import workloads
from workloads.scenes import _prim, default_grid, default_physics


# ---------------------------------------------------------------- geometry
def _inside_fn(scene, P):
    """Implicit surface function used by brute-force marching (sign changes);
    evaluated on an array of points q[..., 3]."""
    c = np.array(P["center"])
    u = np.array(P["u"])
    v = np.array(P["v"])
    n = np.cross(u, v)
    k = P["kind"]
    if k == "box":
        lo, hi = np.array(scene.box_lo), np.array(scene.box_hi)
        return lambda q: np.min(np.minimum(q - lo, hi - q), axis=-1)
    if k in ("rect", "disc"):
        return lambda q: (q - c) @ n
    if k == "cylinder":
        def f(q):
            w = q - c
            return np.linalg.norm(w - np.outer(w @ u, u), axis=-1) - P["p0"]
        return f
    raise ValueError(k)


def _on_patch(scene, P, q):
    c = np.array(P["center"])
    u = np.array(P["u"])
    v = np.array(P["v"])
    k = P["kind"]
    if k == "box":
        return True
    if k == "rect":
        return abs((q - c) @ u) <= P["p0"] and abs((q - c) @ v) <= P["p1"]
    if k == "disc":
        r = math.hypot((q - c) @ u, (q - c) @ v)
        return P["p0"] <= r <= P["p1"]
    return abs((q - c) @ u) <= P["p1"]


def _brute_first_hit(scene, p, d, ell, exclude, steps=40_000):
    ts = np.linspace(0, ell, steps + 1)
    best = (math.inf, -1)
    for li, P in enumerate(scene.prims):
        if li == exclude:
            continue
        f = _inside_fn(scene, P)
        vals = f(p[None, :] + ts[:, None] * d[None, :])
        if P["kind"] == "box":
            idx = np.nonzero(vals <= 0)[0]
            idx = idx[idx > 0]
        else:
            idx = np.nonzero(np.sign(vals[1:]) != np.sign(vals[:-1]))[0] + 1
        for j in idx:
            q = p + ts[j] * d
            if _on_patch(scene, P, q):
                if ts[j] < best[0]:
                    best = (ts[j], li)
                break
    return best


def test_hit_test_matches_brute_force(oracle_mod):
    sc = workloads.scene_quaternary(n_per_cathode=1)
    o = oracle_mod.OracleScene(sc)
    rng = np.random.default_rng(1)
    checked = 0
    for trial in range(60):
        p = rng.uniform([-150, -150, -60], [150, 150, 180])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        ell = rng.uniform(10, 300)
        who, t = o.hit(0, p, d, ell)
        bt, bwho = _brute_first_hit(sc, p, d, ell, -1, steps=8000)
        step = ell / 8000
        if bwho < 0:
            assert who < 0
            continue
        # the marcher resolves t to one step; ambiguous only within a step of an edge
        assert who == bwho or abs(t - bt) < 2 * step, (trial, who, bwho, t, bt)
        assert abs(t - bt) <= 2 * step
        checked += 1
    assert checked > 20


def test_hit_exclusion_and_ties(oracle_mod):
    sc = workloads.scene_single_ni(n=1)
    o = oracle_mod.OracleScene(sc)
    # from the target surface going up: first flight excludes the target itself
    who, t = o.hit(0, [5.0, 0.0, 0.0], [0.0, 0.0, 1.0], 1e9, exclude=1)
    assert who == 4 and abs(t - 100.0) < 1e-12     # substrate rect
    # going down from just above the target: hits it
    who, t = o.hit(0, [5.0, 0.0, 1.0], [0.0, 0.0, -1.0], 1e9)
    assert who == 1 and abs(t - 1.0) < 1e-12
    # segment too short: no hit
    who, t = o.hit(0, [5.0, 0.0, 1.0], [0.0, 0.0, 1.0], 50.0)
    assert who == -1


# ---------------------------------------------------------------- survival
def _open_scene(pressure, L, n, physics):
    """Cosine source in a huge box, a huge plane at height L (no chimney)."""
    big = 1e7
    prims = [_prim("box"),
             _prim("disc", (0, 0, 0), (1, 0, 0), (0, 1, 0), 0.0, 25.4),
             _prim("rect", (0, 0, L), (1, 0, 0), (0, -1, 0), big, big)]
    geoms = [{"prim_begin": 0, "prim_count": 3, "substrate": 2}]
    el = workloads.element("Ni")
    cath = [{"element": el, "center": (0, 0, 0), "normal": (0, 0, 1), "e1": (1, 0, 0),
             "racetrack": {"kind": "gaussian_annulus", "r0": 12.0, "sigma": 3.0, "R": 25.4},
             "cos_coef": (0, 1, 0, 0, 0, 0), "target": 1}]
    inst = [{"geometry": 0, "cathode": 0, "pressure": pressure, "E_i": 400.0, "k": 0.4, "n": n}]
    return workloads.Scene("open", (-big, -big, -big), (big, big, big), workloads.GAS_AR, 300.0, prims,
                           geoms, cath, inst, default_grid(10, 10, 50.0, 50.0), default_physics(**physics), 0)


def test_survival_fraction_exponential_flights(oracle_mod):
    """Constant lambda_m (hard spheres, stationary gas): P(no collision before a
    plane at height L) = int_0^1 2 mu exp(-L/(lambda mu)) dmu = 2 E_3(L/lambda)."""
    d_hs = 3.0
    sigma = math.pi * d_hs**2 * 1e-14                   # mm^2
    L = 40.0
    n_target = 1.0 / (sigma * L)                         # kappa = 1
    p = n_target * 1e9 * 1.380649e-23 * 300.0           # Pa
    n = 20_000
    sc = _open_scene(p, L, n, {"interaction": "hard_sphere", "hs_diameter": d_hs, "gas_motion": "stationary",
                               "max_collisions": 200})
    o = oracle_mod.OracleScene(sc)
    out = o.run_all()
    kappa = o.n_gas(0) * sigma * L
    frac = np.mean((out["prim"] == 2) & (out["ncoll"] == 0))
    want = 2 * special.expn(3, kappa)
    assert abs(frac - want) < 4 * math.sqrt(want * (1 - want) / n), (frac, want)


# ------------------------------------------------------------ vacuum profile
def _view_factor_corner(x, y, h):
    """Diffuse (cosine) emitter to a parallel rectangle [0,x]x[0,y] at height h,
    the corner above the emitter (textbook configuration factor), odd in x, y."""
    X, Y = x / h, y / h
    a, b = math.sqrt(1 + X * X), math.sqrt(1 + Y * Y)
    return (X / a * math.atan(Y / a) + Y / b * math.atan(X / b)) / (2 * math.pi)


def _vacuum_expected(sc, n_r=48, n_phi=96):
    g = sc.grid
    nx, ny, hu, hv = g["nx"], g["ny"], g["half_u"], g["half_v"]
    rt = sc.cathodes[0]["racetrack"]
    r0, sg, R = rt["r0"], rt["sigma"], rt["R"]
    h = 100.0
    xr, wr = np.polynomial.legendre.leggauss(n_r)
    rr = 0.5 * R * (xr + 1)
    wr = 0.5 * R * wr * rr * np.exp(-((rr - r0) ** 2) / (2 * sg * sg))
    wr /= wr.sum()
    phis = 2 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
    ue = np.linspace(-hu, hu, nx + 1)
    ve = np.linspace(-hv, hv, ny + 1)
    F = np.zeros((ny, nx))
    for r, w in zip(rr, wr):
        for ph in phis:
            xs, ys = r * math.cos(ph), r * math.sin(ph)
            us, vs = xs, -ys                                # substrate axes u = +x, v = -y
            cu = np.array([[_view_factor_corner(a - us, b - vs, h) for a in ue] for b in ve])
            F += w / n_phi * (cu[1:, 1:] - cu[1:, :-1] - cu[:-1, 1:] + cu[:-1, :-1])
    return F


@pytest.mark.slow
def test_vacuum_line_of_sight_profile(oracle_mod):
    """p = 0: deposition on the parallel substrate equals the cosine-law view
    factor integrated over the racetrack (chi-square over cells)."""
    n = 60_000
    sc = workloads.scene_single_ni(n=n, pressure=0.0, nx=10, ny=10)
    o = oracle_mod.OracleScene(sc)
    out = o.run_all()
    assert np.all(out["ncoll"] == 0)
    counts = oracle_mod.tally(sc, out)["counts"][0].reshape(10, 10)
    exp = n * _vacuum_expected(sc)
    assert exp.min() > 5
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert stats.chi2.sf(chi2, exp.size) > 1e-3, chi2


# ------------------------------------------------------------ conservation
def test_integer_conservation_and_chunking(oracle_mod):
    """Every particle lands on exactly one primitive or times out; results do
    not depend on how the id range is split (keyed random streams)."""
    sc = workloads.scene_quaternary(n_per_cathode=150)
    o = oracle_mod.OracleScene(sc)
    out = o.run_all(n_threads=3)
    t = oracle_mod.tally(sc, out)
    assert t["prim_counts"].sum() + t["timed_out"].sum() == sc.total_particles
    # re-run a shuffled subset one id at a time
    rng = np.random.default_rng(0)
    sel = rng.choice(len(out["pid"]), 40, replace=False)
    sub = o.run_ids(out["inst"][sel], out["pid"][sel], n_threads=1)
    for k in ("prim", "cell", "ncoll"):
        assert np.array_equal(sub[k], out[k][sel])
    assert np.array_equal(sub["E"], out["E"][sel])


def test_collision_cap_counts_timed_out(oracle_mod):
    sc = workloads.scene_single_ni(n=300, physics={"max_collisions": 2})
    o = oracle_mod.OracleScene(sc)
    out = o.run_all()
    assert out["ncoll"].max() <= 2
    t = oracle_mod.tally(sc, out)
    assert t["timed_out"][0] > 0
    assert t["prim_counts"].sum() + t["timed_out"].sum() == 300


def test_trace_agrees_with_the_outcome(oracle_mod):
    """The per-flight trace (used for GPU trace parity) ends where the particle's
    outcome says: the landing primitive, the collision count, the arrival energy,
    and a path whose collided flights join end to start."""
    sc = workloads.scene_single_ni(n=40)
    osc = oracle_mod.OracleScene(sc)
    out = osc.run_all()
    m_ni = sc.cathodes[0]["element"].mass
    for pid in range(40):
        tr = osc.trace(0, pid, rows=4096)
        status = tr[:, 7]
        last = int(np.nonzero(status >= 0)[0].max())
        if out["prim"][pid] >= 0:
            assert status[last] == 1 and int(tr[last, 8]) == out["prim"][pid]
        else:
            assert status[last] == 2
        assert np.sum(status[1:last] == 0) == out["ncoll"][pid]
        E = 0.5 * m_ni * tr[last, 6] ** 2 * oracle_mod.c_energy()
        assert abs(E - out["E"][pid]) < 1e-9 * out["E"][pid]
        for r in range(1, last):
            # row r holds the collision point of flight r: row r-1 position + t * direction of row r-1
            step = tr[r - 1, :3] + tr[r, 9] * tr[r - 1, 3:6]
            assert np.allclose(step, tr[r, :3], atol=1e-9 * (1 + np.abs(step).max()))


def test_rng_stream_gives_common_random_numbers(oracle_mod):
    """sput_instance.rng_stream: 0 draws the instance's own stream (its index), s > 0 the
    stream s - 1; two instances on the same stream and conditions transport the same
    particle ids identically, and a different stream gives different trajectories."""
    sc = workloads.scene_quaternary(n_per_cathode=300)
    base = oracle_mod.OracleScene(sc).run_all()
    # instance 2 on instance 0's stream with instance 0's cathode and geometry
    sc2 = workloads.scene_quaternary(n_per_cathode=300)
    sc2.instances[2] = dict(sc2.instances[0], rng_stream=1)
    sc2.instances[0] = dict(sc2.instances[0], rng_stream=1)
    sc2.instances[1] = dict(sc2.instances[1], rng_stream=2)     # its own index + 1: unchanged
    o = oracle_mod.OracleScene(sc2).run_all()
    a, b, c = slice(0, 300), slice(300, 600), slice(600, 900)
    for k in ("prim", "cell", "ncoll"):
        assert np.array_equal(o[k][a], base[k][a]) and np.array_equal(o[k][c], base[k][a])
        assert np.array_equal(o[k][b], base[k][b])
    assert np.array_equal(o["E"][c], base["E"][a])
    # instance 3 left on its own stream differs from instance 0's particles
    assert not np.array_equal(base["ncoll"][slice(900, 1200)], base["ncoll"][a])
