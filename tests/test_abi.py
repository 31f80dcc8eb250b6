"""The C-ABI library builds for sm_103a, loads, exports every entry point of
include/sput.h, and its Python mirror has the same struct layouts.  No compute
call is made here (no GPU needed)."""

import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import workloads
from paper_2411_14413_gb300 import _native as N
from paper_2411_14413_gb300 import api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sput.h")


@pytest.fixture(scope="module")
def lib():
    N.build()
    return N.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sput_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "sput_run" in names and "sput_scene_create" in names
    for path in (N.LIB_PATH, N.CHECKED_LIB_PATH):
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
        exported = set(re.findall(r"\bT (sput_\w+)", out))
        missing = [n for n in names if n not in exported]
        assert not missing, (path, missing)
    for n in names:
        assert hasattr(lib, n)
    assert set(names) == set(N.SIGNATURES), set(names) ^ set(N.SIGNATURES)


_LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "sput.h"
#define S(T) printf(#T " %zu\n", sizeof(T));
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  S(sput_chamber) S(sput_primitive) S(sput_geometry) S(sput_cathode) S(sput_instance) S(sput_grid)
  S(sput_physics) S(sput_scene_desc) S(sput_record) S(sput_tallies) S(sput_tally_layout) S(sput_run_opts)
  S(sput_run_stats) S(sput_tune_result) S(sput_microbench_result)
  O(sput_tune_result, cand_rate) O(sput_run_opts, flags)
  O(sput_scene_desc, chamber) O(sput_scene_desc, prims) O(sput_scene_desc, grid) O(sput_scene_desc, physics)
  O(sput_cathode, rt_r0) O(sput_cathode, cos_coef) O(sput_cathode, launch_table) O(sput_cathode, n_E)
  O(sput_cathode, E_hi) O(sput_instance, n_particles) O(sput_instance, rng_stream) O(sput_grid, e_hist_max)
  O(sput_physics, max_collisions) O(sput_physics, thermal_switch_eV) O(sput_run_opts, timeout_ms) O(sput_run_stats, kernel_ms)
  O(sput_tally_layout, n_tickets) O(sput_record, score) O(sput_tallies, score_T)
  return 0;
}
"""


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "lay.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-std=c11", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, lines):
        key, val = line.rsplit(" ", 1)
        if "." in key:
            t, f = key.split(".")
            assert getattr(getattr(N, t), f).offset == int(val), key
        else:
            assert C.sizeof(getattr(N, key)) == int(val), key


def test_version_and_status_strings(lib):
    assert lib.sput_version() == N.SPUT_ABI_VERSION
    assert lib.sput_status_str(0) == b"ok"
    assert lib.sput_status_str(2) == b"invalid scene"


def _create(scene):
    d, keep = api.scene_desc(scene)
    h = C.c_void_p()
    return N.load().sput_scene_create(C.byref(d), 0, C.byref(h))


@pytest.mark.parametrize("mutate,expect", [
    (lambda s: s.instances[0].__setitem__("cathode", 5), 2),
    (lambda s: s.geometries[0].__setitem__("substrate", 99), 2),
    (lambda s: s.prims[2].__setitem__("p0", -1.0), 2),
    (lambda s: s.prims[1].__setitem__("u", (2.0, 0.0, 0.0)), 2),
    (lambda s: s.physics.__setitem__("max_attempts", 0), 2),
    (lambda s: s.physics.__setitem__("chi_min_deg", 0.0), 2),
    (lambda s: s.instances[0].__setitem__("E_i", -5.0), 2),
    (lambda s: s.instances[0].__setitem__("n", 2**32), 2),
    (lambda s: s.cathodes[0].__setitem__("target", 2), 2),
    (lambda s: s.cathodes[0].__setitem__("launch_table", {"weights": np.zeros((4, 4)), "E_hi": 100.0}), 2),
    (lambda s: s.cathodes[0].__setitem__("launch_table", {"weights": -np.ones((4, 4)), "E_hi": 100.0}), 2),
    (lambda s: s.cathodes[0].__setitem__("launch_table", {"weights": np.ones((4, 4)), "E_hi": 0.0}), 2),
    (lambda s: s.cathodes[0].__setitem__("launch_table", {"weights": np.ones((300, 4)), "E_hi": 100.0}), 2),
    (lambda s: s.cathodes[0].__setitem__("launch_table", {"weights": np.full((4, 4), np.nan), "E_hi": 100.0}), 2),
    (lambda s: s.physics.__setitem__("thermal_switch_eV", -1.0), 2),
    (lambda s: s.physics.update({"thermal_switch_eV": 0.1, "gas_motion": "stationary"}), 2),
    # degenerate conditions of the method: no Thompson support (k Lambda E_i <= U_s), a
    # negative or undefined pressure, no head-on factor, a gas at or below 0 K
    (lambda s: s.instances[0].__setitem__("E_i", 5.0), 2),
    (lambda s: s.instances[0].__setitem__("pressure", -0.1), 2),
    (lambda s: s.instances[0].__setitem__("pressure", float("nan")), 2),
    (lambda s: s.instances[0].__setitem__("k", 0.0), 2),
    (lambda s: setattr(s, "T", 0.0), 2),
])
def test_host_validation_rejects_bad_scenes(lib, mutate, expect):
    """Invalid descriptions fail in host validation, before any CUDA call."""
    sc = workloads.scene_single_ni(n=10)
    mutate(sc)
    assert _create(sc) == expect
    assert len(lib.sput_last_error()) > 0


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.sput_scene_create(None, 0, C.byref(h)) == 1
    assert lib.sput_run(None, None, None, None, None) == 1
    assert lib.sput_probe(None, 0, 0, 1, None, None) == 1
    lib.sput_scene_destroy(None)


def test_ion_energy_from_table_s1_voltage_lines(lib):
    """sput_ion_energy (host only): at the two Table S1 powers of each element's supply
    the ion energy equals the tabulated voltage (singly charged ions: E_i/eV = V/volt),
    midway it is their mean, and the line extrapolates; bad lines are rejected."""
    from workloads.measurement import voltage_points

    syms = ("Ni", "Pd", "Pt", "Ru")
    volt = np.array([[*voltage_points(s)[0], *voltage_points(s)[1]] for s in syms], dtype=np.float64)
    out = np.zeros(4)
    for col_p, col_v in ((0, 1), (2, 3)):
        pw = np.ascontiguousarray(volt[:, col_p])
        assert lib.sput_ion_energy(4, volt.ctypes.data, pw.ctypes.data, out.ctypes.data) == 0
        assert np.array_equal(out, volt[:, col_v])
    pw = np.ascontiguousarray(0.5 * (volt[:, 0] + volt[:, 2]))
    assert lib.sput_ion_energy(4, volt.ctypes.data, pw.ctypes.data, out.ctypes.data) == 0
    assert np.allclose(out, 0.5 * (volt[:, 1] + volt[:, 3]), rtol=1e-14)
    pw = np.ascontiguousarray(2 * volt[:, 2] - volt[:, 0])  # one line length beyond P_b
    assert lib.sput_ion_energy(4, volt.ctypes.data, pw.ctypes.data, out.ctypes.data) == 0
    assert np.allclose(out, 2 * volt[:, 3] - volt[:, 1], rtol=1e-13)
    bad = volt.copy()
    bad[1, 2] = bad[1, 0]
    assert lib.sput_ion_energy(4, bad.ctypes.data, pw.ctypes.data, out.ctypes.data) == 1
    assert lib.sput_ion_energy(0, volt.ctypes.data, pw.ctypes.data, out.ctypes.data) == 1
    assert lib.sput_ion_energy(4, None, pw.ctypes.data, out.ctypes.data) == 1
