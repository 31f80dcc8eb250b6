"""Pins for the oracle's random-number stream and launch samplers.

Each test compares the oracle against something other than its own formula:
PyTorch's independent Philox engine, integrals done by scipy, or moments
derived in closed form from the paper's distributions.
"""

import math
import os
import subprocess

import numpy as np
import pytest
from scipy import integrate, stats

import workloads


# --------------------------------------------------------------- Philox
_PH_SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char** argv) {
  for (int a = 1; a + 2 < argc; a += 3) {
    unsigned long long seed = strtoull(argv[a], 0, 0), off = strtoull(argv[a + 1], 0, 0),
                       sub = strtoull(argv[a + 2], 0, 0);
    at::Philox4_32 e(seed, sub, off);
    for (int i = 0; i < 4; i++) printf("%u ", e());
    printf("\n");
  }
}
"""


@pytest.fixture(scope="module")
def torch_philox(tmp_path_factory):
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PyTorch Philox header not installed")
    d = tmp_path_factory.mktemp("ph")
    src = d / "ph.cpp"
    src.write_text(_PH_SRC)
    exe = d / "ph"
    subprocess.run(["g++", "-std=c++17", "-O1", f"-I{inc}", str(src), "-o", str(exe)], check=True)
    return str(exe)


def test_philox_matches_pytorch_engine(oracle_mod, torch_philox):
    """Philox4x32-10 (Salmon et al., SC'11) against PyTorch's own engine.
    PyTorch maps key = seed (lo, hi) and counter = (offset lo, offset hi,
    subsequence lo, subsequence hi)."""
    rng = np.random.default_rng(7)
    cases = [(0, 0, 0)] + [tuple(int(x) for x in rng.integers(0, 2**63, 3)) for _ in range(40)]
    cases.append((2**64 - 1, 2**64 - 1, 2**64 - 1))
    args = []
    for s, o, q in cases:
        args += [str(s), str(o), str(q)]
    lines = subprocess.run([torch_philox] + args, check=True, capture_output=True, text=True).stdout.split("\n")
    for (s, o, q), line in zip(cases, lines):
        ref = [int(x) for x in line.split()]
        got = oracle_mod.philox([o & 0xFFFFFFFF, o >> 32, q & 0xFFFFFFFF, q >> 32], [s & 0xFFFFFFFF, s >> 32])
        assert list(map(int, got)) == ref, (s, o, q)


def test_uniform_mapping_open_closed(oracle_mod):
    """RN_1 must lie in ]0,1] (Eq. for lambda): 0 maps to 2^-24, 2^32-1 to 1."""
    u = oracle_mod.uniform_from_word([0, 255, 256, 2**32 - 1])
    assert u[0] == 2.0**-24 and u[1] == 2.0**-24 and u[2] == 2.0 * 2.0**-24 and u[3] == 1.0


def test_quadrature_self_check(oracle_mod):
    assert abs(oracle_mod.integrate_test(0, 0.0, 1.0) - (math.e - 1)) < 1e-14
    assert abs(oracle_mod.integrate_test(1, 0.0, 1.0) - math.pi / 4) < 1e-14
    assert abs(oracle_mod.integrate_test(2, 0.0, 1.0) - 2.0 / 3.0) < 1e-12


# --------------------------------------------------------------- Thompson
def _thompson_mean_closed_form(Em, U):
    # <E> = int_0^Em E^2/(E+U)^3 dE / int_0^Em E/(E+U)^3 dE, both by hand:
    # num = ln((Em+U)/U) + 2U/(Em+U) - U^2/(2(Em+U)^2) - 3/2
    # den = Em^2 / (2U(Em+U)^2)
    num = math.log((Em + U) / U) + 2 * U / (Em + U) - U * U / (2 * (Em + U) ** 2) - 1.5
    den = Em * Em / (2 * U * (Em + U) ** 2)
    return num / den


@pytest.mark.parametrize("sym", ["Ni", "Pd", "Pt", "Ru"])
def test_thompson_emax_and_mean(oracle_mod, sym):
    """E_max = k Lambda E_i - U_s with Lambda the head-on energy-transfer
    fraction 1 - ((M_i-M_t)/(M_i+M_t))^2 (same quantity as 4 M_i M_t/(M_i+M_t)^2);
    the sampler's mean over a fine u grid equals the closed-form mean."""
    el = workloads.element(sym)
    Mi, Mt = workloads.GAS_AR.mass, el.mass
    lam = 1.0 - ((Mi - Mt) / (Mi + Mt)) ** 2
    Em = oracle_mod.emax(0.4, Mi, Mt, 400.0, el.U_s)
    assert abs(Em - (0.4 * lam * 400.0 - el.U_s)) < 1e-12
    n = 200_000
    u = (np.arange(n) + 0.5) / n
    E = np.array([oracle_mod.thompson(Em, el.U_s, x) for x in u[:: n // 20_000]])
    # exact endpoints of the inverse CDF
    assert abs(oracle_mod.thompson(Em, el.U_s, 1.0) - Em) < 1e-9 * Em
    assert oracle_mod.thompson(Em, el.U_s, 1e-30) < 1e-6
    # mean: midpoint rule in u of E(u); E(u) ~ sqrt(u) near 0, so use a change of variables u = t^2
    m = 40_000
    t = (np.arange(m) + 0.5) / m
    Et = np.array([oracle_mod.thompson(Em, el.U_s, x * x) for x in t])
    mean = np.sum(Et * 2 * t) / m
    assert abs(mean - _thompson_mean_closed_form(Em, el.U_s)) < 2e-4 * mean
    assert np.all(np.diff(E) > 0)


def test_thompson_distribution_ks(oracle_mod):
    """KS test of sampled energies against phi(E) ~ E/(E+U)^3 on [0,E_max]
    integrated numerically by scipy (not the closed-form CDF)."""
    U, Em = 4.44, 149.78
    norm = integrate.quad(lambda e: e / (e + U) ** 3, 0, Em, epsabs=1e-14, epsrel=1e-13)[0]

    def cdf(x):
        x = np.atleast_1d(x)
        return np.array([integrate.quad(lambda e: e / (e + U) ** 3, 0, min(max(v, 0), Em))[0] / norm for v in x])

    rng = np.random.default_rng(3)
    u = rng.uniform(0, 1, 3000)
    E = np.array([oracle_mod.thompson(Em, U, x) for x in u])
    assert stats.kstest(E, cdf).pvalue > 1e-3


# ----------------------------------------------------------- cosine sum
def test_cosine_moments(oracle_mod):
    """Pure cosine (c_1 = 1): <mu> = 2/3, <mu^2> = 1/2 (pdf in mu ~ mu)."""
    n = 20_000
    u = (np.arange(n) + 0.5) / n
    mu = np.array([oracle_mod.cos_mu([0, 1, 0, 0, 0, 0], x) for x in u])
    assert abs(mu.mean() - 2 / 3) < 1e-4
    assert abs((mu**2).mean() - 0.5) < 1e-4
    # closed form inverse of the cosine case is sqrt(u)
    assert np.max(np.abs(mu - np.sqrt(u))) < 1e-12


@pytest.mark.parametrize("coef", [(1, 0, 0, 0, 0, 0), (0.2, 0.5, 0.1, 0.0, 0.3, 0.05), (0, 0, 0, 0, 0, 1)])
def test_cosine_sum_moments(oracle_mod, coef):
    """General six-term sum: <mu^k> = sum c_i/(i+k+1) / sum c_i/(i+1)."""
    n = 20_000
    u = (np.arange(n) + 0.5) / n
    mu = np.array([oracle_mod.cos_mu(list(coef), x) for x in u])
    den = sum(c / (i + 1) for i, c in enumerate(coef))
    for k in (1, 2, 3):
        want = sum(c / (i + k + 1) for i, c in enumerate(coef)) / den
        assert abs((mu**k).mean() - want) < 5e-4, k


# ------------------------------------------------------------- racetrack
def test_racetrack_cdf_and_moments(oracle_mod):
    """Radial pdf ~ r d(r) with d a Gaussian annulus (r0=12, sigma=3) on [0, 25.4]:
    the oracle's CDF and inverse agree with scipy quadrature of r d(r)."""
    r0, sg, R = 12.0, 3.0, 25.4
    f = lambda r: r * math.exp(-((r - r0) ** 2) / (2 * sg * sg))
    Z = integrate.quad(f, 0, R, epsabs=0, epsrel=1e-13)[0]
    for r in [0.5, 5.0, 11.0, 12.0, 15.5, 20.0, 25.0]:
        want = integrate.quad(f, 0, r, epsabs=0, epsrel=1e-13)[0] / Z
        assert abs(oracle_mod.racetrack_cdf(r0, sg, R, r) - want) < 1e-11
    mean_want = integrate.quad(lambda r: r * f(r), 0, R, epsrel=1e-13)[0] / Z
    m2_want = integrate.quad(lambda r: r * r * f(r), 0, R, epsrel=1e-13)[0] / Z
    n = 20_000
    u = (np.arange(n) + 0.5) / n
    rr = np.array([oracle_mod.racetrack_r(r0, sg, R, x) for x in u])
    assert abs(rr.mean() - mean_want) < 2e-4
    assert abs((rr**2).mean() - m2_want) < 5e-3
    assert rr.min() >= 0 and rr.max() <= R
    assert abs(oracle_mod.racetrack_r(r0, sg, R, 1.0) - R) < 1e-9


# ------------------------------------------------- joint (mu, E) launch table
def _table_scene(weights, E_hi):
    return workloads.scene_single_ni_table(n=1, table={"weights": np.asarray(weights, float), "E_hi": E_hi})


def _table_samples(oracle_mod, weights, E_hi, n=20000, seed=1):
    osc = oracle_mod.OracleScene(_table_scene(weights, E_hi))
    rng = np.random.default_rng(seed)
    u = 1.0 - rng.random((n, 2))          # ]0, 1]
    out = np.array([osc.table_launch(0, a, b) for a, b in u])
    osc.close()
    return out[:, 0], out[:, 1]


def _piecewise_cdf(cell_weights, width):
    """CDF of the piecewise-uniform density with the given cell weights."""
    w = np.asarray(cell_weights, float)
    F = np.concatenate([[0.0], np.cumsum(w)]) / w.sum()

    def cdf(x):
        j = np.clip((np.asarray(x) / width).astype(int), 0, len(w) - 1)
        t = np.clip(np.asarray(x) / width - j, 0.0, 1.0)
        return F[j] + t * (F[j + 1] - F[j])
    return cdf


def test_launch_table_uniform_table_gives_uniform_mu_and_E(oracle_mod):
    mu, E = _table_samples(oracle_mod, np.ones((8, 16)), 100.0)
    assert stats.kstest(mu, "uniform").pvalue > 1e-3
    assert stats.kstest(E / 100.0, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(mu, E)[0, 1]) < 4 / math.sqrt(len(mu))


def test_launch_table_single_cell(oracle_mod):
    w = np.zeros((8, 16))
    w[3, 5] = 2.5
    mu, E = _table_samples(oracle_mod, w, 160.0, n=4000)
    assert np.all((mu > 3 / 8) & (mu <= 4 / 8)) and np.all((E > 50.0) & (E <= 60.0))
    assert stats.kstest((mu - 3 / 8) * 8, "uniform").pvalue > 1e-3
    assert stats.kstest((E - 50.0) / 10.0, "uniform").pvalue > 1e-3


def test_launch_table_marginals_and_conditional(oracle_mod):
    """Synthetic table with mu-E correlation: the mu marginal and the E marginal
    follow the exact piecewise-linear CDFs of the table; the energies drawn in
    the top and the bottom mu cell have their rows' exact means."""
    t = workloads.synthetic_launch_table(n_mu=16, n_E=32, E_hi=120.0)
    w, E_hi = t["weights"], t["E_hi"]
    mu, E = _table_samples(oracle_mod, w, E_hi, n=30000)
    assert stats.kstest(mu, _piecewise_cdf(w.sum(1), 1 / 16)).pvalue > 1e-3
    dE = E_hi / 32
    # E marginal: mixture over rows of piecewise-uniform densities = piecewise uniform with column sums
    assert stats.kstest(E, _piecewise_cdf(w.sum(0), dE)).pvalue > 1e-3
    centres = (np.arange(32) + 0.5) * dE
    for i in (0, 15):
        sel = (mu > i / 16) & (mu <= (i + 1) / 16)
        want = (w[i] * centres).sum() / w[i].sum()
        second = (w[i] * (centres ** 2 + dE ** 2 / 12)).sum() / w[i].sum()
        sd = math.sqrt(second - want ** 2)
        assert abs(E[sel].mean() - want) < 4 * sd / math.sqrt(sel.sum()), (i, E[sel].mean(), want)
    # the high-energy tail is more forward-peaked than the low-energy part
    assert mu[E > 60].mean() > mu[E < 5].mean()


def test_launch_table_cell_edges(oracle_mod):
    """u equal to a cumulative weight ends the cell exactly (t = 1); cells of
    zero weight are never drawn."""
    w = np.array([[1.0, 0.0, 3.0], [0.0, 0.0, 0.0], [2.0, 2.0, 0.0]])
    osc = oracle_mod.OracleScene(_table_scene(w, 30.0))
    mu, E = osc.table_launch(0, 4.0 / 8.0, 0.25)       # end of mu cell 0; E: end of E cell 0
    assert mu == pytest.approx(1 / 3) and E == pytest.approx(10.0)
    mu, E = osc.table_launch(0, 4.0 / 8.0 + 1e-9, 1.0)  # just past cell 0 -> cell 2 (cell 1 empty)
    assert mu > 2 / 3 and E == pytest.approx(20.0)
    osc.close()


# ------------------------------------------- derivative with respect to E_max
def test_thompson_cutoff_derivative_identity(oracle_mod):
    """For the Thompson law on (0, E_max], d P(E > E0)/dE_max equals
    p(E_max) (1 - P(E > E0)), p(E_max) = 2U/(E_max (E_max + U)): the LR term
    -p(E_max) E[f] plus the moving-support term p(E_max) f(E_max).  Checked
    against central differences of the normalised CDF by quadrature."""
    U = 4.44

    def p_above(E0, Em):
        dens = lambda e: e / (e + U) ** 3
        Z = integrate.quad(dens, 0.0, Em, epsabs=0, epsrel=1e-13)[0]
        return integrate.quad(dens, E0, Em, epsabs=0, epsrel=1e-13)[0] / Z

    for Em in (20.0, 149.78):
        # p(E_max) is the normalised density at the cut-off
        Z = integrate.quad(lambda e: e / (e + U) ** 3, 0.0, Em, epsabs=0, epsrel=1e-13)[0]
        pE = 2 * U / (Em * (Em + U))
        assert abs(Em / (Em + U) ** 3 / Z - pE) < 1e-12 * pE
        for E0 in (1.0, 5.0, 0.5 * Em):
            h = 1e-4 * Em
            fd = (p_above(E0, Em + h) - p_above(E0, Em - h)) / (2 * h)
            assert abs(fd - pE * (1 - p_above(E0, Em))) < 1e-7 * pE, (Em, E0)


def test_oracle_launch_at_cutoff(oracle_mod):
    """The boundary run changes only the launch energy: E = E_max, same point and direction."""
    sc = workloads.scene_single_ni(n=10)
    o = oracle_mod.OracleScene(sc)
    Em = o.emax(0)
    for pid in range(5):
        p, d, E = o.launch(0, pid)
        o.set_at_cutoff(True)
        pc, dc, Ec = o.launch(0, pid)
        o.set_at_cutoff(False)
        assert np.array_equal(p, pc) and np.array_equal(d, dc)
        assert E < Em and Ec == Em
