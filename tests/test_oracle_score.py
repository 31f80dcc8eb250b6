"""CPU pins of the oracle's pressure score S = d ln p(path)/d ln n_g.

Pressure enters the path density only through the free flights (Eq. for
lambda): a flight of length l that ends in a collision contributes
1 - l/lambda, the last flight, cut short by the surface at distance t,
contributes -t/lambda.  These tests pin the oracle's per-particle score
against the mathematics, not against the CUDA path:

* closed form: for a constant mean free path (hard spheres, gas at rest) and
  a cosine source, the probability of reaching a plane at height L without a
  collision is 2 E_3(kappa), kappa = n sigma L, so its derivative in ln p is
  -2 kappa E_2(kappa).  The likelihood-ratio estimate is mean(1{no collision,
  on the plane} S).  The test also shows that a score scaled by 1.05, by 2 or
  with its sign flipped would fail it.
* common random numbers: the score's estimate of d P(land in a region)/d ln p
  over whole multi-collision trajectories agrees with central finite
  differences of the oracle's own landing fractions (same seed, p e^{+-h}).
"""

import math

import numpy as np
from scipy import special

import workloads
from workloads import ELEMENTS
from workloads.scenes import _prim, default_grid, default_physics

KB = 1.380649e-23


def _slab_scene(n, d_hs, L, kappa, T=300.0):
    """Cathode disc at z = 0 facing +z, an infinite plane at z = L, gas at rest,
    hard spheres of diameter d_hs (Angstrom); pressure chosen so that n sigma L = kappa;
    one flight per atom (max_collisions = 0: an atom that collides is retired)."""
    sigma = math.pi * d_hs**2 * 1e-14  # mm^2
    p = kappa / (sigma * L) * 1e9 * KB * T
    big = 1e7
    prims = [_prim("box"), _prim("disc", (0, 0, 0), (1, 0, 0), (0, 1, 0), 0.0, 25.4),
             _prim("rect", (0, 0, L), (1, 0, 0), (0, -1, 0), big, big)]
    cath = [{"element": ELEMENTS["Ni"], "center": (0, 0, 0), "normal": (0, 0, 1), "e1": (1, 0, 0),
             "racetrack": {"kind": "gaussian_annulus", "r0": 12.0, "sigma": 3.0, "R": 25.4},
             "cos_coef": (0, 1, 0, 0, 0, 0), "target": 1}]
    return workloads.Scene("slab", (-big, -big, -big), (big, big, big), workloads.GAS_AR, T, prims,
                           [{"prim_begin": 0, "prim_count": 3, "substrate": 2}], cath,
                           [{"geometry": 0, "cathode": 0, "pressure": p, "E_i": 400.0, "k": 0.4, "n": n}],
                           default_grid(4, 4, 50.0, 50.0),
                           default_physics(interaction="hard_sphere", hs_diameter=d_hs, gas_motion="stationary",
                                           max_collisions=0), 0)


def test_score_survival_derivative_closed_form(oracle_mod):
    n, kappa = 1_000_000, 1.0
    sc = _slab_scene(n, 3.0, 40.0, kappa)
    o = oracle_mod.OracleScene(sc).run_all()
    f = ((o["prim"] == 2) & (o["ncoll"] == 0)).astype(float)
    # the uncollided fraction itself: 2 E_3(kappa)
    assert abs(f.mean() - 2 * special.expn(3, kappa)) < 4 * f.std() / math.sqrt(n)
    # on an uncollided path to the plane the score is -t/lambda = -kappa/mu
    s = o["score"]
    est = f * s
    want = -2 * kappa * special.expn(2, kappa)
    tol = 4 * est.std() / math.sqrt(n)
    assert abs(est.mean() - want) < tol, (est.mean(), want, tol)
    # the test has the power to see a wrong scale or sign of the score
    for wrong in (1.05, 2.0, -1.0):
        assert abs(wrong * est.mean() - want) > tol, wrong
    # atoms that collided carry 1 - l/lambda with l < the distance to the plane
    coll = o["prim"] < 0
    assert coll.any() and np.all(s[coll] <= 1.0)


def _chamber_hs_scene(n, pressure):
    return workloads.scene_single_ni(n=n, pressure=pressure, nx=10, ny=10,
                                     physics={"interaction": "hard_sphere", "hs_diameter": 3.0,
                                              "gas_motion": "stationary"})


def test_score_matches_crn_finite_difference(oracle_mod):
    n, p0, h = 600_000, 0.5, 0.15
    sc = _chamber_hs_scene(n, p0)
    sub = sc.geometries[0]["substrate"]
    o = oracle_mod.OracleScene(sc).run_all()
    assert o["ncoll"].mean() > 1.0  # multi-collision trajectories

    # region: the central 6 x 6 of the 10 x 10 substrate cells
    def in_region(out):
        c = out["cell"]
        return (out["prim"] == sub) & (c >= 0) & (c % 10 >= 2) & (c % 10 < 8) & (c // 10 >= 2) & (c // 10 < 8)

    r0 = in_region(o).astype(float)
    lr = r0 * o["score"]
    fr = []
    for sgn in (+1, -1):
        out = oracle_mod.OracleScene(_chamber_hs_scene(n, p0 * math.exp(sgn * h))).run_all()
        fr.append(in_region(out).astype(float))
    fd = (fr[0] - fr[1]) / (2 * h)
    # standard error of the difference of the two estimates (paired: same particles)
    diff = lr - fd
    se = diff.std() / math.sqrt(n)
    # central differences carry an O(h^2) bias: bound it by the third derivative of a
    # survival-like exp(-c p) curve, |f'''| h^2 / 6 <= 0.01 |f'| for these h and c
    bias = 0.01 * abs(fd.mean())
    assert abs(lr.mean() - fd.mean()) < 4 * se + bias, (lr.mean(), fd.mean(), se)
    assert abs(fd.mean()) > 8 * se  # the derivative is resolved
    for wrong in (2.0, -1.0):
        assert abs(wrong * lr.mean() - fd.mean()) > 4 * se + bias, wrong
