"""Pins for the oracle's interaction physics: scattering angle, cross section,
mean free path, collision kinematics and partner weighting (Sec. "The SIMTRA
model": elastic collisions with neutral gas atoms in thermal equilibrium under
a screened-Coulomb potential with Moliere screening)."""

import math

import numpy as np
import pytest
from scipy import integrate, special, stats

import workloads

CHI_MIN = math.radians(1.0)
MOL_C = (0.35, 0.55, 0.10)
MOL_D = (0.3, 1.2, 6.0)


# ------------------------------------------------------------ scattering angle
@pytest.mark.parametrize("eps", [1e-8, 1e-5, 1e-3, 0.1, 1.0, 30.0])
@pytest.mark.parametrize("beta", [0.01, 0.3, 2.0, 17.0, 400.0])
def test_chi_coulomb_is_rutherford(oracle_mod, eps, beta):
    """Unscreened Coulomb (Phi = 1): tan(chi/2) = Z1 Z2 e^2 / (2 E_r b) = 1/(2 eps beta)."""
    got = oracle_mod.chi(eps, beta, "coulomb")
    want = 2.0 * math.atan(1.0 / (2.0 * eps * beta))
    assert abs(got - want) < 1e-11 * max(1.0, want)


def test_chi_head_on_and_monotone(oracle_mod):
    for eps in [1e-7, 1e-4, 1e-2, 1.0]:
        assert abs(oracle_mod.chi(eps, 1e-9) - math.pi) < 1e-6
        betas = np.geomspace(1e-3, 200, 60)
        chis = [oracle_mod.chi(eps, b) for b in betas]
        assert all(a > b for a, b in zip(chis, chis[1:]))
        assert all(0 < c <= math.pi for c in chis)


def test_chi_impulse_approximation(oracle_mod):
    """For large impact parameters the deflection approaches the impulse
    approximation chi = (1/eps) sum c_i d_i K1(d_i beta); the relative gap
    must shrink as chi -> 0."""
    for eps in [1e-6, 1e-4, 1e-2]:
        gaps = []
        bm = oracle_mod.bmax_direct(eps, CHI_MIN)
        for f in [1.5, 2.5, 4.0, 6.0]:
            beta = bm * f
            chi = oracle_mod.chi(eps, beta)
            imp = sum(c * d * special.k1(d * beta) for c, d in zip(MOL_C, MOL_D)) / eps
            gaps.append(abs(chi - imp) / imp)
        assert gaps[-1] < 0.01, gaps
        # shrinking until it reaches the rounding floor
        assert all(a > b or b < 1e-13 for a, b in zip(gaps, gaps[1:])), gaps


@pytest.mark.parametrize("eps,beta", [(1e-3, 10.0), (1e-3, 25.0), (1e-6, 40.0), (0.1, 0.5), (2.0, 0.2)])
def test_chi_against_arbitrary_precision(oracle_mod, eps, beta):
    """The classical deflection integral evaluated independently in 40-digit
    arithmetic (mpmath): apsis by bracketed root finding on
    g(x) = 1 - beta^2/x^2 - Phi(x)/(eps x), then with x = x0/u
    chi = pi - 2 (beta/x0) int_0^1 du / sqrt(1 - (beta u/x0)^2 - u Phi(x0/u)/(eps x0))
    by tanh-sinh quadrature, which handles the end-point singularity at u = 1."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    e, b = mp.mpf(eps), mp.mpf(beta)
    phi = lambda x: sum(mp.mpf(c) * mp.exp(-mp.mpf(d) * x) for c, d in zip(MOL_C, MOL_D))
    g = lambda x: 1 - (b / x) ** 2 - phi(x) / (e * x)
    hi = (1 / e + mp.sqrt(1 / e**2 + 4 * b * b)) / 2
    x0 = mp.findroot(g, (b, hi * (1 + mp.mpf(10) ** -30)), solver="anderson")
    assert abs(oracle_mod.x0(eps, beta) - float(x0)) < 1e-13 * float(x0)
    F = lambda u: 1 - (b * u / x0) ** 2 - u * phi(x0 / u) / (e * x0)
    I = mp.quad(lambda u: 1 / mp.sqrt(F(u)), [0, mp.mpf("0.5"), 1])
    want = float(mp.pi - 2 * b / x0 * I)
    assert abs(oracle_mod.chi(eps, beta) - want) < 1e-11 * max(want, 1e-3), (oracle_mod.chi(eps, beta), want)


def test_hard_sphere_chi(oracle_mod):
    """Hard spheres: b = d cos(chi/2)."""
    for b in [0.0, 0.1, 0.5, 0.9, 1.0]:
        assert abs(math.cos(oracle_mod.chi_hard_sphere(b) / 2) - b) < 1e-14


# ------------------------------------------------------------ cross section
@pytest.mark.parametrize("eps", [1e-4, 1e-2, 1.0, 50.0])
def test_bmax_coulomb_closed_form(oracle_mod, eps):
    """Angle cut-off cross section: in the Coulomb limit b_max = 1/(2 eps tan(chi_min/2))."""
    got = oracle_mod.bmax_direct(eps, CHI_MIN, "coulomb")
    want = 1.0 / (2 * eps * math.tan(CHI_MIN / 2))
    assert abs(got - want) < 1e-10 * want


def test_bmax_lagrange_cache_matches_direct_root(oracle_mod):
    rng = np.random.default_rng(11)
    for le in rng.uniform(-38.0, 4.0, 25):
        e = math.exp(le)
        a, b = oracle_mod.bmax_interp(e, CHI_MIN), oracle_mod.bmax_direct(e, CHI_MIN)
        assert abs(a - b) < 1e-10 * b, (le, a, b)
        assert abs(oracle_mod.chi(e, b) - CHI_MIN) < 1e-12


def test_cross_section_values_ni_ar(oracle_mod):
    """sigma(E_r) = pi b_max^2 at the 1 deg cut-off decreases with energy and
    is of the size of a few atomic radii squared; a_F(Ni-Ar) from the Firsov
    formula 0.8853 a0 (Z1^1/2 + Z2^1/2)^-2/3."""
    sc = workloads.scene_single_ni(n=1)
    o = oracle_mod.OracleScene(sc)
    a = o.a_screen(0)
    assert abs(a - 0.8853 * 0.529177210903 * (math.sqrt(28) + math.sqrt(18)) ** (-2 / 3)) < 1e-14
    mu = 58.6934 * 39.948 / (58.6934 + 39.948)
    ce = oracle_mod.c_energy()
    sig = []
    for Er in [0.01, 0.1, 1.0, 10.0, 100.0]:
        g = math.sqrt(2 * Er / (mu * ce))
        sig.append(o.sigma(0, g))
    assert all(x > y for x, y in zip(sig, sig[1:]))
    assert 10.0 < sig[-1] < 40.0 and 40.0 < sig[2] < 80.0


# ------------------------------------------------------------ mean free path
def _mean_rel_speed(v, s):
    """<|v - V|> for V ~ Maxwellian with per-axis std s (textbook closed form)."""
    if v == 0:
        return 2.0 * s * math.sqrt(2.0 / math.pi)
    x = v / s
    return s * (math.sqrt(2 / math.pi) * math.exp(-x * x / 2) + (x + 1 / x) * math.erf(x / math.sqrt(2)))


def test_relative_speed_pdf(oracle_mod):
    s = 0.25
    for v in [0.0, 1e-6, 0.1, 0.5, 3.0, 12.0]:
        lo, hi = max(0.0, v - 14 * s), v + 14 * s
        Z = integrate.quad(lambda g: oracle_mod.rel_speed_pdf(g, v, s), lo, hi, epsabs=1e-13, limit=200)[0]
        m = integrate.quad(lambda g: g * oracle_mod.rel_speed_pdf(g, v, s), lo, hi, epsabs=1e-13, limit=200)[0]
        assert abs(Z - 1) < 1e-10
        assert abs(m - _mean_rel_speed(v, s)) < 1e-9


def test_K_hard_sphere_closed_form(oracle_mod):
    """Hard spheres in a thermal gas: <sigma g> = pi d^2 <|v - V|>."""
    sc = workloads.scene_single_ni(n=1, physics={"interaction": "hard_sphere", "hs_diameter": 3.0})
    o = oracle_mod.OracleScene(sc)
    s = o.s_gas()
    assert abs(s - math.sqrt(8.617333262e-5 * 300 / (39.948 * oracle_mod.c_energy()))) < 1e-14
    for v in [0.0, 0.05, 0.3, 1.0, 5.0, 20.0]:
        want = math.pi * 9.0 * _mean_rel_speed(v, s)
        assert abs(o.K(0, v) - want) < 1e-10 * want
        # lambda_m = v / (n_g <sigma g>), n_g = p / (k_B T)
        if v > 0:
            n_mm3 = 0.5 / (1.380649e-23 * 300.0) * 1e-9
            assert abs(o.lam(0, v) - v / (n_mm3 * want * 1e-14)) < 1e-9 * o.lam(0, v)


def test_K_stationary_limit(oracle_mod):
    """Stationary gas: lambda_m = 1/(n_g sigma(v))."""
    sc = workloads.scene_single_ni(n=1, physics={"gas_motion": "stationary"})
    o = oracle_mod.OracleScene(sc)
    n_mm3 = o.n_gas(0)
    for v in [0.3, 2.0, 9.0]:
        assert abs(o.lam(0, v) * n_mm3 * o.sigma(0, v) * 1e-14 - 1.0) < 1e-12


ENV_M = 2.0 * math.sqrt(2.0 / math.pi)   # mean speed / s of the Maxwellian (chi, 3 degrees of freedom)


def test_envelope_bounds_h(oracle_mod):
    """The rejection envelope A + B rho >= sigma(g) g for every relative speed g that a
    partner of speed rho s can give (g^2 = v^2 + s^2 rho^2 - 2 v s rho cos), rho <= 8,
    and it is nearly tight at rho = E[rho] (the upper hull of a concave bound)."""
    sc = workloads.scene_quaternary(n_per_cathode=1)
    o = oracle_mod.OracleScene(sc)
    s = o.s_gas()
    for c in range(4):
        for v in [1e-3, 0.2, 0.5, 1.0, 4.0, 15.0]:
            A, B = o.envelope(c, v)
            assert A >= 0 and B >= 0
            for rho in np.linspace(0.0, 8.0, 65):
                for cs in np.linspace(-1.0, 1.0, 21):
                    g = math.sqrt(max(v * v + s * s * rho * rho - 2 * v * s * rho * cs, 1e-18))
                    assert o.sigma(c, g) * g <= (A + B * rho) * (1 + 1e-12), (c, v, rho, cs)
            gm = np.linspace(max(0.0, v - s * ENV_M), v + s * ENV_M, 400)[1:]
            Hm = max(o.sigma(c, g) * g for g in gm)
            assert A + B * ENV_M <= 1.01 * Hm, (c, v, A + B * ENV_M, Hm)


@pytest.mark.parametrize("v", [0.3, 1.2, 6.0])
def test_partner_law_and_mean_attempts(oracle_mod, v):
    """Partners drawn for an atom of speed v (km/s): the relative speed g = |v - V|
    follows sigma(g) g times the Maxwellian relative-speed density (KS test against
    the quadrature CDF), the mean partner velocity along v matches the 2-D quadrature
    of the weighted Maxwellian, and the mean number of attempts is (A + B E[rho]) / K(v)."""
    sc = workloads.scene_single_ni(n=1)
    o = oracle_mod.OracleScene(sc)
    s = o.s_gas()
    n = 12000
    vv = np.array([0.0, 0.0, v])
    Vs, att = [], []
    for pid in range(n):
        V, a = o.partner(0, pid, 5, vv)
        Vs.append(V)
        att.append(a)
    Vs, att = np.array(Vs), np.array(att, float)
    g = np.linalg.norm(vv - Vs, axis=1)
    h = lambda x: o.sigma(0, x) * x
    grid = np.linspace(1e-9, v + 9 * s, 3001)
    pdf = np.array([h(x) * oracle_mod.rel_speed_pdf(x, v, s) for x in grid])
    cdf = integrate.cumulative_trapezoid(pdf, grid, initial=0)
    K = cdf[-1]
    assert abs(K / o.K(0, v) - 1) < 1e-3
    p_ks = stats.kstest(g, lambda x: np.interp(x, grid, cdf / K)).pvalue
    assert p_ks > 1e-3, p_ks
    # mean of V along v: int f(V) h(|v - V|) V_par dV / K, V = s rho (sin, 0, cos)
    f = lambda r, c: (r * r * math.exp(-0.5 * r * r) / math.sqrt(2 * math.pi) * 2 / 2)
    num = integrate.dblquad(lambda c, r: f(r, c) * h(math.sqrt(max(v * v + s * s * r * r - 2 * v * s * r * c, 1e-18)))
                            * s * r * c, 0, 9, -1, 1, epsabs=1e-10, epsrel=1e-8)[0]
    den = integrate.dblquad(lambda c, r: f(r, c) * h(math.sqrt(max(v * v + s * s * r * r - 2 * v * s * r * c, 1e-18))),
                            0, 9, -1, 1, epsabs=1e-10, epsrel=1e-8)[0]
    want_par = num / den
    got = Vs[:, 2]
    assert abs(got.mean() - want_par) < 4 * got.std() / math.sqrt(n), (got.mean(), want_par)
    A, B = o.envelope(0, v)
    want_att = (A + B * ENV_M) / o.K(0, v)
    assert 1.0 <= want_att < 2.0
    assert abs(att.mean() - want_att) < 4 * att.std() / math.sqrt(n) + 1e-3, (att.mean(), want_att)


# ------------------------------------------------------------ kinematics
def test_collision_invariants(oracle_mod):
    """Elastic collision: momentum, kinetic energy and |g| conserved."""
    sc = workloads.scene_quaternary(n_per_cathode=1)
    o = oracle_mod.OracleScene(sc)
    rng = np.random.default_rng(5)
    mg = 39.948
    for c in range(4):
        m1 = sc.cathodes[c]["element"].mass
        for _ in range(20):
            v = rng.normal(0, 3, 3)
            V = rng.normal(0, 0.3, 3)
            vo, Vo, chi = o.collide(c, v, V, rng.uniform(1e-6, 1), rng.uniform(0, 1))
            assert np.allclose(m1 * v + mg * V, m1 * vo + mg * Vo, rtol=0, atol=1e-12)
            e0 = m1 * v @ v + mg * V @ V
            assert abs(m1 * vo @ vo + mg * Vo @ Vo - e0) < 1e-12 * e0
            assert abs(np.linalg.norm(vo - Vo) - np.linalg.norm(v - V)) < 1e-12
            g0, g1 = v - V, vo - Vo
            assert abs(math.acos(np.clip(g0 @ g1 / (g0 @ g0), -1, 1)) - chi) < 1e-6


def test_hard_sphere_uniform_energy_loss(oracle_mod):
    """Hard spheres, target at rest: the lab energy after one collision is
    uniform on [E ((m1-m2)/(m1+m2))^2, E], linear in the uniform u_b."""
    sc = workloads.scene_single_ni(n=1, physics={"interaction": "hard_sphere"})
    o = oracle_mod.OracleScene(sc)
    m1, m2 = 58.6934, 39.948
    alpha = ((m1 - m2) / (m1 + m2)) ** 2
    v = np.array([0.0, 0.0, 5.0])
    E0 = v @ v
    for ub in np.linspace(0.0, 1.0, 21):
        vo, _, _ = o.collide(0, v, np.zeros(3), ub, 0.3)
        want = alpha + (1 - alpha) * ub
        assert abs(vo @ vo / E0 - want) < 1e-12


def _thermal_check(oracle_mod, physics, n_particles, n_coll, burn, stride, pmin, plant=False):
    sc = workloads.scene_single_ni(n=1, physics=physics)
    o = oracle_mod.OracleScene(sc)
    if plant:
        o.plant_unweighted_partner()
    m1, mg = 58.6934, 39.948
    kT = 8.617333262e-5 * 300.0
    ce = oracle_mod.c_energy()
    sm = math.sqrt(kT / (m1 * ce))       # per-axis std of the sputtered atom at equilibrium
    samples = []
    for pid in range(n_particles):
        sp = o.thermalize(0, pid, 20.0, n_coll)
        samples.append(sp[burn::stride])
    samples = np.concatenate(samples)
    # jump-chain stationary law: speed density ~ v^2 exp(-v^2/(2 sm^2)) * nu(v), nu = n <sigma g>
    vmax = 12 * sm
    dens = lambda v: v * v * math.exp(-v * v / (2 * sm * sm)) * o.K(0, v)
    grid = np.linspace(0, vmax, 801)
    pdf = np.array([dens(x) for x in grid])
    cdf = integrate.cumulative_trapezoid(pdf, grid, initial=0)
    cdf /= cdf[-1]
    return stats.kstest(samples, lambda x: np.interp(x, grid, cdf)).pvalue


@pytest.mark.slow
def test_thermalisation_hard_sphere(oracle_mod):
    """Partner weighting: after many collisions the post-collision speeds follow
    the collision-weighted Maxwellian of the sputtered mass at the gas T."""
    p = _thermal_check(oracle_mod, {"interaction": "hard_sphere"}, 60, 400, 100, 10, 1e-3)
    assert p > 1e-3


@pytest.mark.slow
def test_thermalisation_moliere(oracle_mod):
    p = _thermal_check(oracle_mod, {}, 48, 600, 200, 40, 1e-3)
    assert p > 1e-3


@pytest.mark.slow
def test_thermalisation_detects_an_unweighted_partner(oracle_mod):
    """Planted mistake: the partner drawn from the plain Maxwellian, without the
    sigma(g) g weighting; the thermalisation test must reject it."""
    p = _thermal_check(oracle_mod, {"interaction": "hard_sphere"}, 60, 400, 100, 10, 1e-3, plant=True)
    assert p < 1e-3, p
