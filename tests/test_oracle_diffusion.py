"""Pins for the oracle's diffusion shortcut for thermalised atoms: the
momentum-transfer and diffusion cross sections against closed forms and an
independent integration, and the pressure score of the random walk."""

import math

import numpy as np
from scipy import integrate

import workloads


def test_hard_sphere_cross_sections_closed_form(oracle_mod):
    """Hard spheres scatter isotropically in the CM frame, so sigma_m = pi d^2, and the
    first Chapman-Enskog diffusion coefficient gives sigma_D = (32/9) d^2 sqrt(mu/m1)."""
    d = 3.0
    sc = workloads.scene_single_ni(n=1, physics={"interaction": "hard_sphere", "hs_diameter": d,
                                                 "thermal_switch_eV": 0.1})
    o = oracle_mod.OracleScene(sc)
    for g in (0.1, 1.0, 7.0):
        assert abs(o.sigma_m(0, g) - math.pi * d * d) < 1e-12
    m1, m2 = sc.cathodes[0]["element"].mass, workloads.GAS_AR.mass
    want = 32.0 / 9.0 * d * d * math.sqrt(m2 / (m1 + m2))
    assert abs(o.sigma_D(0) - want) < 1e-8 * want


def test_sigma_m_moliere_independent_integration(oracle_mod):
    """sigma_m = 2 pi a^2 int (1 - cos chi) beta dbeta by scipy's adaptive quadrature
    over the oracle's (separately pinned) deflection function."""
    sc = workloads.scene_single_ni(n=1, physics={"thermal_switch_eV": 0.1})
    o = oracle_mod.OracleScene(sc)
    a = o.a_screen(0)
    m1, m2 = sc.cathodes[0]["element"].mass, workloads.GAS_AR.mass
    mu = m1 * m2 / (m1 + m2)
    zze2 = 28 * 18 * 14.3996454784
    for g in (0.3, 1.0, 4.0):
        eps = a * 0.5 * mu * g * g * oracle_mod.c_energy() / zze2
        f = lambda b: 2 * math.sin(0.5 * oracle_mod.chi(eps, b)) ** 2 * b
        B = 400.0
        assert oracle_mod.chi(eps, B) < 1e-9
        val = sum(integrate.quad(f, B * k / 40, B * (k + 1) / 40, epsabs=0, epsrel=1e-10, limit=200)[0]
                  for k in range(40))
        want = 2 * math.pi * a * a * val
        assert abs(o.sigma_m(0, g) - want) < 1e-7 * want, (g, o.sigma_m(0, g), want)
        # a screened potential transfers less momentum than its chi_min-cut total cross section counts
        assert o.sigma_m(0, g) < o.sigma(0, g)


def test_walk_pressure_score_has_zero_mean(oracle_mod):
    """The random walk's step rate n sigma_D is proportional to the pressure: the
    score keeps zero mean with the shortcut on (3 Pa, most atoms thermalise)."""
    sc = workloads.scene_single_ni(n=1500, pressure=3.0, physics={"thermal_switch_eV": 0.1})
    o = oracle_mod.OracleScene(sc).run_all()
    s = o["score"]
    assert np.all(np.isfinite(s)) and o["ncoll"].mean() > 20
    assert abs(s.mean()) < 4 * s.std() / math.sqrt(len(s)), (s.mean(), s.std())
