"""The library's deflection table (host evaluation of the same bicubic cells the
device reads, through the C ABI, no GPU) against the oracle's FP64 deflection
of the Moliere potential (adaptive quadrature of the classical scattering
integral, pinned to Rutherford, the impulse approximation and a 40-digit
evaluation in test_oracle_physics.py).  The table is built from the library's
own FP64 deflection, so this is a parity check of product host code against the
oracle; the bound 5e-7 rad is the FP32 rounding level of a deflection near pi."""

import ctypes as C
import math

import numpy as np
import pytest

from paper_2411_14413_gb300 import _native as N


@pytest.fixture(scope="module")
def lib():
    N.build()
    return N.load()


def _table_chi(lib, chi_min, eps, u):
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(len(eps))
    rc = lib.sput_deflection_table_eval(chi_min, len(eps), eps.ctypes.data_as(C.c_void_p),
                                        u.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p))
    assert rc == 0, lib.sput_last_error()
    return out


def test_table_matches_oracle_deflection(lib, oracle_mod):
    chi_min = math.radians(1.0)
    rng = np.random.default_rng(7)
    n = 4000
    le = rng.uniform(-25.9, -2.1, n)
    # b = b_max sqrt(u): half the points uniform in u (as collisions draw them), half
    # uniform in ln s down to the table's lower edge
    u = np.where(np.arange(n) % 2 == 0, rng.uniform(1e-9, 1.0, n), np.exp(2 * rng.uniform(-5.99, 0.0, n)))
    got = _table_chi(lib, chi_min, np.exp(le), u)
    want = np.array([oracle_mod.chi(math.exp(x), oracle_mod.bmax_interp(math.exp(x), chi_min) * math.sqrt(w))
                     for x, w in zip(le, u)])
    err = np.abs(got - want)
    assert err.max() < 5e-7, (err.max(), le[err.argmax()], u[err.argmax()])
    # at b = b_max the deflection is chi_min by the definition of the cross section
    edge = _table_chi(lib, chi_min, np.exp(np.array([-20.0, -12.3, -4.0])), np.ones(3))
    assert np.allclose(edge, chi_min, rtol=0, atol=1e-9)


def test_outside_the_table_falls_back_to_the_integral(lib, oracle_mod):
    """ln eps outside [-26, -2] or ln s below -6: the FP64 integral, the same function
    the device integrates there."""
    chi_min = math.radians(1.0)
    eps = np.array([math.exp(-30.0), math.exp(-1.0), math.exp(-10.0)])
    u = np.array([0.3, 0.3, math.exp(-13.0)])
    got = _table_chi(lib, chi_min, eps, u)
    want = np.array([oracle_mod.chi(e, oracle_mod.bmax_interp(e, chi_min) * math.sqrt(w)) for e, w in zip(eps, u)])
    assert np.max(np.abs(got - want)) < 1e-8, (got, want)


def test_bad_arguments_are_rejected(lib):
    one = np.ones(1)
    zero = np.zeros(1)
    assert lib.sput_deflection_table_eval(0.0, 1, one.ctypes.data, one.ctypes.data, one.ctypes.data) == 1
    assert lib.sput_deflection_table_eval(0.01, 1, zero.ctypes.data, one.ctypes.data, one.ctypes.data) == 1
    assert lib.sput_deflection_table_eval(0.01, 1, one.ctypes.data, zero.ctypes.data, one.ctypes.data) == 1
