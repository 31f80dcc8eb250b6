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
