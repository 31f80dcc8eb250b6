"""Pins for the oracle's temperature score d ln p(path)/dT (pressure fixed).

T enters the path density through n_g = p/(k_B T) in the collision rate
n_g K(v)/v and through the gas partner density f_T(V) sigma(g) g / K(v), whose
Maxwellian spread is s = sqrt(k_B T / m_gas)."""

import math

import numpy as np

import workloads


def _dlnmean_dlns_closed(v, s):
    """d ln <|v - V|> / d ln s for V ~ N(0, s^2 I): the textbook mean relative
    speed differentiated symbolically."""
    import sympy as sp

    vv, ss = sp.symbols("v s", positive=True)
    m = ss * sp.sqrt(2 / sp.pi) * sp.exp(-vv ** 2 / (2 * ss ** 2)) + (vv + ss ** 2 / vv) * sp.erf(vv / (sp.sqrt(2) * ss))
    expr = sp.diff(m, ss) * ss / m
    return float(expr.subs({vv: v, ss: s}).evalf(30))


def test_dlnK_dlns_hard_sphere_closed_form(oracle_mod):
    sc = workloads.scene_single_ni(n=1, physics={"interaction": "hard_sphere", "hs_diameter": 3.0})
    o = oracle_mod.OracleScene(sc)
    s = o.s_gas()
    for v in [0.05, 0.3, 1.0, 5.0, 20.0]:
        want = _dlnmean_dlns_closed(v, s)
        assert abs(o.dlnK_dlns(0, v) - want) < 1e-7 * max(1.0, abs(want)), (v, o.dlnK_dlns(0, v), want)


def test_partner_spread_matches_dlnK(oracle_mod):
    """The accepted partner density q(V) = f_T(V) sigma(g) g / K(v) integrates
    to one at every T, so E_q[d ln f_T/dT] = d ln K/dT, i.e.
    E_q[|V|^2 / s^2] = 3 + d ln K/d ln s: ties the sampler, its weighting and
    the derivative of K together (Moliere pair, thermal gas)."""
    sc = workloads.scene_single_ni(n=1)
    o = oracle_mod.OracleScene(sc)
    s = o.s_gas()
    for v in [0.2, 1.0, 6.0]:
        x = np.array([np.dot(V, V) / s ** 2 for V, _ in (o.partner(0, pid, 1, [0.0, 0.0, v]) for pid in range(40000))])
        want = 3.0 + o.dlnK_dlns(0, v)
        assert abs(x.mean() - want) < 4 * x.std() / math.sqrt(len(x)), (v, x.mean(), want)


def test_temperature_score_stationary_gas_is_minus_pressure_score_over_T(oracle_mod):
    """Gas at rest: T acts only through n_g = p/(k_B T), so d/dT = -(1/T) d/d ln n_g."""
    sc = workloads.scene_single_ni(n=300, physics={"gas_motion": "stationary", "max_collisions": 150})
    o = oracle_mod.OracleScene(sc).run_all(score_T=True)
    assert np.allclose(o["score_T"], -o["score"] / sc.T, rtol=1e-9, atol=1e-12)


def test_temperature_score_has_zero_mean(oracle_mod):
    """The path density integrates to one at every T: E[score_T] = 0."""
    sc = workloads.scene_single_ni(n=3000, physics={"max_collisions": 40})
    o = oracle_mod.OracleScene(sc).run_all(score_T=True)
    st = o["score_T"]
    assert np.all(np.isfinite(st)) and st.std() > 0
    assert abs(st.mean()) < 4 * st.std() / math.sqrt(len(st)), (st.mean(), st.std())
