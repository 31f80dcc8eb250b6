"""Build and load libsput.so (the CUDA transport library) and mirror its C ABI.

The library is compiled in-tree with nvcc for sm_103a only.  Loading never
falls back to anything else: if the shared object is missing and cannot be
built, or no CUDA device is present when a compute call is made, an error is
raised.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
CSRC = os.path.join(_PKG, "csrc")
INCLUDE = os.path.join(_ROOT, "include")
BUILD = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(BUILD, "libsput.so")
CHECKED_LIB_PATH = os.path.join(BUILD, "libsput_checked.so")
CHECKED_SOURCE = "sput_transport.cu"
SOURCES = ["sput_api.cpp", "sput_tables.cpp", "sput_transport.cu", "sput_adjoint.cu", "sput_microbench.cu"]
HEADERS = ["sput_internal.h", "sput_tables.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

_lock = threading.Lock()
_lib = None


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.{cpp,cu} for sm_103a (in parallel) and link libsput.so, and
    libsput_checked.so: the same library with the transport kernel built with
    SPUT_CHECKED (every table, cell, primitive and record index tested against its
    buffer, a failure reported in the run's status word)."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "sput.h")]
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{CSRC}"]

    def compile_one(job):
        src, checked = job
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + (".checked.o" if checked else ".o"))
        if force or _stale(o, [s] + headers):
            cmd = [nvcc] + common + (["-DSPUT_CHECKED"] if checked else []) + ["-c", s, "-o", o]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            if verbose:
                print(r.stdout + r.stderr)
        return o

    jobs = [(src, False) for src in SOURCES] + [(CHECKED_SOURCE, True)]
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    regular = objs[:len(SOURCES)]
    checked = [objs[-1] if SOURCES[i] == CHECKED_SOURCE else regular[i] for i in range(len(SOURCES))]
    for lib_path, lib_objs in ((LIB_PATH, regular), (CHECKED_LIB_PATH, checked)):
        if force or _stale(lib_path, lib_objs):
            tmp = lib_path + f".tmp{os.getpid()}"
            r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + lib_objs, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
            os.replace(tmp, lib_path)
    return LIB_PATH


# --------------------------------------------------------------- ABI mirror
SPUT_ABI_VERSION = 5
SPUT_OK = 0
STATUS_NAMES = {0: "SPUT_OK", 1: "SPUT_ERR_INVALID_ARG", 2: "SPUT_ERR_INVALID_SCENE", 3: "SPUT_ERR_CUDA",
                4: "SPUT_ERR_TIMEOUT", 5: "SPUT_ERR_DEVICE_CHECK", 6: "SPUT_ERR_UNSUPPORTED", 7: "SPUT_ERR_NO_MEMORY"}
PRIM_KIND = {"box": 0, "rect": 1, "disc": 2, "cylinder": 3}
INTERACTION = {"moliere": 0, "hard_sphere": 1}
GAS_MOTION = {"thermal": 0, "stationary": 1}
COUNT_TYPE = {"int32": 0, "int64": 1}
PROBE = {"chi": 0, "bmax": 1, "K": 2, "M": 3, "launch": 4, "trace": 5, "chi_u": 6}
TRACE_ROWS = 64

D3 = C.c_double * 3


class sput_chamber(C.Structure):
    _fields_ = [("box_lo", D3), ("box_hi", D3), ("gas_Z", C.c_int), ("reserved", C.c_int),
                ("gas_mass", C.c_double), ("gas_T", C.c_double)]


class sput_primitive(C.Structure):
    _fields_ = [("kind", C.c_int), ("reserved", C.c_int), ("center", D3), ("u", D3), ("v", D3),
                ("p0", C.c_double), ("p1", C.c_double)]


class sput_geometry(C.Structure):
    _fields_ = [("prim_begin", C.c_int), ("prim_count", C.c_int), ("substrate", C.c_int), ("reserved", C.c_int)]


class sput_cathode(C.Structure):
    _fields_ = [("Z", C.c_int), ("target", C.c_int), ("mass", C.c_double), ("U_s", C.c_double),
                ("center", D3), ("normal", D3), ("e1", D3),
                ("rt_r0", C.c_double), ("rt_sigma", C.c_double), ("rt_R", C.c_double),
                ("cos_coef", C.c_double * 6),
                ("launch_table", C.POINTER(C.c_double)), ("n_mu", C.c_int), ("n_E", C.c_int), ("E_hi", C.c_double)]


class sput_instance(C.Structure):
    _fields_ = [("geometry", C.c_int), ("cathode", C.c_int), ("pressure", C.c_double), ("E_i", C.c_double),
                ("k", C.c_double), ("n_particles", C.c_uint64), ("rng_stream", C.c_uint32), ("reserved", C.c_uint32)]


class sput_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("half_u", C.c_double), ("half_v", C.c_double),
                ("count_type", C.c_int), ("n_ebins", C.c_int), ("e_hist_max", C.c_double),
                ("n_abins", C.c_int), ("reserved", C.c_int)]


class sput_physics(C.Structure):
    _fields_ = [("chi_min", C.c_double), ("hs_diameter", C.c_double), ("interaction", C.c_int),
                ("gas_motion", C.c_int), ("max_attempts", C.c_int), ("reserved", C.c_int),
                ("max_collisions", C.c_int64), ("thermal_switch_eV", C.c_double)]


class sput_scene_desc(C.Structure):
    _fields_ = [("abi_version", C.c_uint32), ("n_prims", C.c_int), ("n_geoms", C.c_int), ("n_cathodes", C.c_int),
                ("n_instances", C.c_int), ("chamber", sput_chamber), ("prims", C.POINTER(sput_primitive)),
                ("geoms", C.POINTER(sput_geometry)), ("cathodes", C.POINTER(sput_cathode)),
                ("instances", C.POINTER(sput_instance)), ("grid", sput_grid), ("physics", sput_physics)]


class sput_record(C.Structure):
    _fields_ = [("prim", C.c_int32), ("cell", C.c_int32), ("energy", C.c_float), ("cos_angle", C.c_float),
                ("n_collisions", C.c_uint32), ("score", C.c_float)]


class sput_tallies(C.Structure):
    _fields_ = [("counts", C.c_void_p), ("energy", C.c_void_p), ("score", C.c_void_p),
                ("prim_counts", C.c_void_p), ("timed_out", C.c_void_p), ("hist_E", C.c_void_p),
                ("hist_A", C.c_void_p), ("records", C.c_void_p), ("score_T", C.c_void_p)]


class sput_tally_layout(C.Structure):
    _fields_ = [("n_instances", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("max_prims", C.c_int),
                ("n_ebins", C.c_int), ("n_abins", C.c_int), ("count_type", C.c_int), ("reserved", C.c_int),
                ("n_tickets", C.c_uint64)]


class sput_run_opts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("ticket_begin", C.c_uint64), ("ticket_end", C.c_uint64),
                ("accumulate", C.c_int), ("block_threads", C.c_int), ("blocks_per_sm", C.c_int),
                ("ticket_chunk", C.c_int), ("timeout_ms", C.c_int), ("flags", C.c_int)]


class sput_run_stats(C.Structure):
    _fields_ = [("particles", C.c_uint64), ("landed", C.c_uint64), ("timed_out", C.c_uint64),
                ("flights", C.c_uint64), ("collisions", C.c_uint64), ("attempts", C.c_uint64),
                ("device_status", C.c_uint32), ("grid_blocks", C.c_uint32), ("block_threads", C.c_uint32),
                ("kernel_ms", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sput_tune_result(C.Structure):
    _fields_ = [("block_threads", C.c_int), ("blocks_per_sm", C.c_int), ("ticket_chunk", C.c_int),
                ("flags", C.c_int), ("best_rate", C.c_float), ("n_candidates", C.c_int), ("reserved", C.c_int),
                ("cand_threads", C.c_int * 32), ("cand_bps", C.c_int * 32), ("cand_chunk", C.c_int * 32),
                ("cand_flags", C.c_int * 32), ("cand_rate", C.c_float * 32)]

    def candidates(self):
        return [dict(threads=self.cand_threads[i], bps=self.cand_bps[i], chunk=self.cand_chunk[i],
                     flags=self.cand_flags[i], rate=self.cand_rate[i]) for i in range(self.n_candidates)]


class sput_microbench_result(C.Structure):
    _fields_ = [("ops", C.c_double), ("ms", C.c_double), ("ops_per_s", C.c_double), ("blocks", C.c_int),
                ("threads", C.c_int)]


MICROBENCH_KINDS = {"ffma": 0, "mufu_lg2": 1, "mufu_ex2": 2, "mufu_rsqrt": 3, "mufu_sin": 4, "philox": 5,
                    "red_i32": 6, "red_i64": 7, "red_f64": 8}

SPUT_RUN_NO_SMEM_COUNTERS = 1
SPUT_RUN_SMEM_COUNTERS = 2
SPUT_RUN_LAUNCH_AT_CUTOFF = 4
SPUT_RUN_INJECT_NONFINITE = 8
SPUT_RUN_NO_CELL_MASKS = 16
SPUT_RUN_CELL_MASKS = 32

ABI_STRUCTS = [sput_chamber, sput_primitive, sput_geometry, sput_cathode, sput_instance, sput_grid, sput_physics,
               sput_scene_desc, sput_record, sput_tallies, sput_tally_layout, sput_run_opts, sput_run_stats,
               sput_tune_result, sput_microbench_result]

# name -> (restype, argtypes) for every entry point declared in include/sput.h
_P = C.c_void_p
SIGNATURES = {
    "sput_version": (C.c_int, []),
    "sput_status_str": (C.c_char_p, [C.c_int]),
    "sput_last_error": (C.c_char_p, []),
    "sput_scene_create": (C.c_int, [C.POINTER(sput_scene_desc), C.c_int, C.POINTER(_P)]),
    "sput_instances_set": (C.c_int, [_P, C.POINTER(sput_instance), C.c_int]),
    "sput_tally_layout_get": (C.c_int, [_P, C.POINTER(sput_tally_layout)]),
    "sput_run": (C.c_int, [_P, C.POINTER(sput_run_opts), _P, C.POINTER(sput_tallies), C.POINTER(sput_run_stats)]),
    "sput_run_host": (C.c_int, [_P, C.POINTER(sput_run_opts), C.POINTER(sput_tallies), C.POINTER(sput_run_stats)]),
    "sput_run_noalloc": (C.c_int, [_P, C.POINTER(sput_run_opts), _P, C.POINTER(sput_tallies), C.POINTER(sput_run_stats)]),
    "sput_scene_destroy": (None, [_P]),
    "sput_autotune": (C.c_int, [_P, C.POINTER(sput_run_opts), _P, C.POINTER(sput_tallies), C.c_uint64,
                                C.POINTER(sput_tune_result)]),
    "sput_graph_create": (C.c_int, [_P, C.POINTER(sput_run_opts), _P, C.POINTER(sput_tallies), C.POINTER(_P)]),
    "sput_graph_launch": (C.c_int, [_P, C.c_uint64, _P]),
    "sput_graph_destroy": (None, [_P]),
    "sput_backward": (C.c_int, [_P, _P, _P, _P, _P]),
    "sput_emax_backward": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "sput_ion_energy": (C.c_int, [C.c_int, _P, _P, _P]),
    "sput_voltage_backward": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "sput_composition": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, _P, C.c_int, _P, _P, _P, _P, _P]),
    "sput_composition_backward": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, _P, C.c_int, _P, _P, _P, _P, _P, _P,
                                            _P]),
    "sput_probe": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P]),
    "sput_deflection_table_eval": (C.c_int, [C.c_double, C.c_int, _P, _P, _P]),
    "sput_microbench": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, C.c_size_t, C.c_int, _P,
                                  C.POINTER(sput_microbench_result)]),
}


def load(path: str | None = None, build_if_missing: bool = True):
    """Load libsput.so; builds it first when missing or stale (needs nvcc)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if path is None and build_if_missing:
            srcs = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "sput.h")]
            if _stale(p, srcs):
                build()
        if not os.path.exists(p):
            raise RuntimeError(f"libsput.so not found at {p}; run __graft_entry__.build()")
        L = C.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        if path is None:
            _lib = L
        return L


class SputError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.sput_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, where):
    if status != SPUT_OK:
        raise SputError(status, where)
