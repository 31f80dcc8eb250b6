"""FP64 CPU oracle for the sputter-transport hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
``--impl reference`` leg may import this package.  The product path
(``paper_2411_14413_gb300``) never imports it, and the two share no code: the
only shared module is ``workloads`` (seeded scene descriptions without any of
the method's arithmetic).

The transport itself lives in ``sput_oracle.c`` (plain C, double precision,
one particle at a time, pthreads over particle ids).  This module compiles it
with gcc, marshals a ``workloads.Scene`` into the oracle's own flat layouts,
and turns per-particle outcomes into tallies.

Parity status of each oracle function (pins in tests/test_oracle_*.py):
  Philox4x32-10            pinned: PyTorch's independent Philox engine
  Thompson sampler         pinned: closed-form CDF and mean (Eq. for phi(E))
  cosine-sum sampler       pinned: closed-form moments (Eq. for d2Y/dOmega)
  racetrack sampler        pinned: scipy quadrature of r * d(r)
  scattering angle chi     pinned: Rutherford (Coulomb limit), impulse
                           approximation (large b), chi -> pi as b -> 0
  b_max / cross section    pinned: Rutherford cut-off closed form; Lagrange
                           cache vs direct root
  K(v) = <sigma g>         pinned: hard-sphere closed form of <|v - V|>
  free flight + surfaces   pinned: survival fraction 2 E_3(n sigma L) and the
                           vacuum view-factor deposition profile
  collision kinematics     pinned: momentum/energy invariants; hard-sphere
                           uniform energy loss
  partner weighting        pinned: thermalisation to the collision-weighted
                           Maxwellian (and a first-proposal-only partner
                           fails it); the partner's relative-speed law against
                           quadrature of sigma(g) g times the Maxwellian
                           relative-speed density; mean attempts against the
                           envelope's (A + B E[rho]) / K(v); the envelope
                           bounds sigma(g) g over every reachable g
  pressure score (LR)      pinned: d/d ln p of the uncollided fraction,
                           -2 kappa E_2(kappa) (closed form); central
                           finite differences of the landing fractions with
                           common random numbers
  absolute deposition profile under the chi_min cut-off: parity unpinned
  (no printed value in the paper checks it).
"""

from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sput_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsput_oracle.so")
_lib = None
_lock = threading.Lock()

PK = {"box": 0, "rect": 1, "disc": 2, "cylinder": 3}
INTERACTION = {"moliere": 0, "hard_sphere": 1}
GAS_MOTION = {"thermal": 0, "stationary": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: no -march, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC,
           "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i, u64, p = C.c_double, C.c_int, C.c_uint64, C.c_void_p
            L.or_scene_new.restype = p
            L.or_scene_new.argtypes = [p, i, p, i, p, i, p, i, p, p, p]
            L.or_scene_free.argtypes = [p]
            L.or_run_ids.restype = i
            L.or_run_ids.argtypes = [p, u64, C.c_int64, p, p, i, p, p, p, p, p, p, p, p]
            L.or_scene_set_score_T.restype = None
            L.or_scene_set_score_T.argtypes = [p, i]
            L.or_scene_set_at_cutoff.restype = None
            L.or_scene_set_at_cutoff.argtypes = [p, i]
            L.or_scene_plant_unweighted_partner.restype = None
            L.or_scene_plant_unweighted_partner.argtypes = [p, i]
            for name, args in {
                "or_chi": [i, d, d], "or_x0": [i, d, d], "or_chi_hard_sphere": [d],
                "or_bmax_direct": [i, d, d], "or_bmax_interp": [d, d],
                "or_emax": [d, d, d, d, d], "or_racetrack_cdf": [d, d, d, d],
                "or_racetrack_r": [d, d, d, d], "or_thompson": [d, d, d], "or_cos_mu": [p, d],
                "or_c_energy": [], "or_s_gas": [p], "or_n_gas": [p, i], "or_inst_emax": [p, i],
                "or_cath_ascr": [p, i], "or_sigma": [p, i, d], "or_K": [p, i, d],
                "or_lambda": [p, i, d], "or_rel_speed_pdf": [d, d, d], "or_integrate_test": [i, d, d],
                "or_dlnK_dlns": [p, i, d], "or_sigma_m": [p, i, d], "or_sigma_D": [p, i],
            }.items():
                f = getattr(L, name)
                f.restype = d
                f.argtypes = args
            L.or_envelope.restype = None
            L.or_envelope.argtypes = [p, i, d, p, p]
            L.or_cath_monotone.restype = i
            L.or_cath_monotone.argtypes = [p, i]
            L.or_hit.restype = i
            L.or_hit.argtypes = [p, i, p, p, d, i, p]
            L.or_collide.restype = None
            L.or_collide.argtypes = [p, i, p, p, d, d, p, p, p]
            L.or_partner.restype = i
            L.or_partner.argtypes = [p, u64, i, u64, C.c_uint32, p, p]
            L.or_thermalize.restype = None
            L.or_thermalize.argtypes = [p, u64, i, u64, d, i, p]
            L.or_trace.restype = None
            L.or_trace.argtypes = [p, u64, i, u64, i, p]
            L.or_launch.restype = None
            L.or_launch.argtypes = [p, u64, i, u64, p, p, p]
            L.or_philox.restype = None
            L.or_philox.argtypes = [p, p, p]
            L.or_set_launch_table.restype = i
            L.or_set_launch_table.argtypes = [p, i, i, i, d, p]
            L.or_table_launch.restype = None
            L.or_table_launch.argtypes = [p, i, d, d, p, p]
            L.or_version.restype = i
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


# ----------------------------------------------------------- scene marshalling
def _flatten(scene):
    ch = np.array(list(scene.box_lo) + list(scene.box_hi) + [scene.gas.Z, scene.gas.mass, scene.T], float)
    prims = np.zeros((len(scene.prims), 16), float)
    for i, P in enumerate(scene.prims):
        prims[i, 0] = PK[P["kind"]]
        prims[i, 1:4] = P["center"]
        prims[i, 4:7] = P["u"]
        prims[i, 7:10] = P["v"]
        prims[i, 10] = P["p0"]
        prims[i, 11] = P["p1"]
    geoms = np.array([[g["prim_begin"], g["prim_count"], g["substrate"]] for g in scene.geometries], np.int32)
    cath = np.zeros((len(scene.cathodes), 32), float)
    for i, c in enumerate(scene.cathodes):
        el = c["element"]
        rt = c["racetrack"]
        if rt["kind"] != "gaussian_annulus":
            raise ValueError("oracle supports the Gaussian-annulus racetrack only")
        cath[i, 0:3] = [el.Z, el.mass, el.U_s]
        cath[i, 3:6] = c["center"]
        cath[i, 6:9] = c["normal"]
        cath[i, 9:12] = c["e1"]
        cath[i, 12:15] = [rt["r0"], rt["sigma"], rt["R"]]
        cath[i, 15:21] = c["cos_coef"]
        cath[i, 21] = c["target"]
    inst = np.zeros((len(scene.instances), 8), float)
    for i, I in enumerate(scene.instances):
        inst[i, 0:6] = [I["geometry"], I["cathode"], I["pressure"], I["E_i"], I["k"], I.get("rng_stream", 0)]
    g = scene.grid
    grid = np.array([g["nx"], g["ny"], g["half_u"], g["half_v"], g["n_ebins"], g["e_hist_max"],
                     g["n_abins"], 0.0], float)
    ph = scene.physics
    phys = np.array([math.radians(ph["chi_min_deg"]), INTERACTION[ph["interaction"]], ph["hs_diameter"],
                     GAS_MOTION[ph["gas_motion"]], ph["max_attempts"], ph["max_collisions"],
                     ph.get("thermal_switch_eV", 0.0), 0.0], float)
    return ch, prims, geoms, cath, inst, grid, phys


class OracleScene:
    """The oracle's own copy of a workloads.Scene."""

    def __init__(self, scene):
        self.scene = scene
        self._arrays = _flatten(scene)
        ch, prims, geoms, cath, inst, grid, phys = self._arrays
        L = lib()
        self.h = L.or_scene_new(_ptr(ch), len(prims), _ptr(prims), len(geoms), _ptr(geoms),
                                len(cath), _ptr(cath), len(inst), _ptr(inst), _ptr(grid), _ptr(phys))
        if not self.h:
            raise RuntimeError("or_scene_new failed")
        self._tables = []
        for ci, c in enumerate(scene.cathodes):
            lt = c.get("launch_table")
            if lt is None:
                continue
            w = np.ascontiguousarray(lt["weights"], dtype=np.float64)
            self._tables.append(w)
            if L.or_set_launch_table(self.h, ci, w.shape[0], w.shape[1], float(lt["E_hi"]), _ptr(w)) != 0:
                raise RuntimeError("or_set_launch_table failed")

    def close(self):
        if getattr(self, "h", None):
            lib().or_scene_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- per-particle transport ------------------------------------------------
    def run_ids(self, inst_ids, pids, n_threads=None, seed=None, score_T=False, at_cutoff=False):
        """Outcomes of particles (inst_ids[i], pids[i]); score_T adds the
        temperature score (d ln p(path)/dT at fixed pressure; slower);
        at_cutoff launches every atom with E = E_max (boundary run)."""
        inst_ids = np.ascontiguousarray(inst_ids, dtype=np.int32)
        pids = np.ascontiguousarray(pids, dtype=np.uint64)
        n = len(pids)
        out = {
            "prim": np.empty(n, np.int32), "cell": np.empty(n, np.int32), "E": np.empty(n, float),
            "cos": np.empty(n, float), "ncoll": np.empty(n, np.int64), "score": np.empty(n, float),
            "attempts": np.empty(n, np.int64),
        }
        if score_T:
            out["score_T"] = np.empty(n, float)
        if n_threads is None:
            n_threads = os.cpu_count() or 1
        seed = self.scene.seed if seed is None else seed
        L = lib()
        L.or_scene_set_score_T(self.h, 1 if score_T else 0)
        L.or_scene_set_at_cutoff(self.h, 1 if at_cutoff else 0)
        rc = L.or_run_ids(self.h, int(seed), n, _ptr(inst_ids), _ptr(pids), int(n_threads),
                          _ptr(out["prim"]), _ptr(out["cell"]), _ptr(out["E"]), _ptr(out["cos"]),
                          _ptr(out["ncoll"]), _ptr(out["score"]), _ptr(out["attempts"]),
                          _ptr(out["score_T"]) if score_T else None)
        if rc != 0:
            raise ValueError("or_run_ids rejected its inputs")
        out["inst"] = inst_ids
        out["pid"] = pids
        return out

    def run_all(self, n_threads=None, seed=None, score_T=False, at_cutoff=False):
        """Every particle of every instance, in ticket order (instance-major)."""
        ids, pids = [], []
        for i, I in enumerate(self.scene.instances):
            ids.append(np.full(int(I["n"]), i, np.int32))
            pids.append(np.arange(int(I["n"]), dtype=np.uint64))
        return self.run_ids(np.concatenate(ids), np.concatenate(pids), n_threads, seed, score_T, at_cutoff)

    def sigma_m(self, cath, g):
        """Momentum-transfer cross section (Angstrom^2) at relative speed g (km/s)."""
        return lib().or_sigma_m(self.h, int(cath), float(g))

    def sigma_D(self, cath):
        """Diffusion cross section (Angstrom^2) of the shortcut: 1/lambda_D = n sigma_D."""
        return lib().or_sigma_D(self.h, int(cath))

    def dlnK_dlns(self, cath, v):
        """d ln K / d ln s at speed v (s = per-axis thermal spread of the gas)."""
        return lib().or_dlnK_dlns(self.h, int(cath), float(v))

    # -- probes -----------------------------------------------------------------
    def sigma(self, cath, g):
        return lib().or_sigma(self.h, cath, g)

    def K(self, cath, v):
        return lib().or_K(self.h, cath, v)

    def envelope(self, cath, v):
        """(A, B) of the partner-rejection envelope A + B |V|/s at atom speed v (km/s)."""
        A, B = C.c_double(), C.c_double()
        lib().or_envelope(self.h, cath, v, C.byref(A), C.byref(B))
        return A.value, B.value

    def lam(self, inst, v):
        return lib().or_lambda(self.h, inst, v)

    def s_gas(self):
        return lib().or_s_gas(self.h)

    def n_gas(self, inst):
        return lib().or_n_gas(self.h, inst)

    def emax(self, inst):
        return lib().or_inst_emax(self.h, inst)

    def a_screen(self, cath):
        return lib().or_cath_ascr(self.h, cath)

    def monotone(self, cath):
        return lib().or_cath_monotone(self.h, cath)

    def hit(self, geom, p, d, ell, exclude=-1):
        p = np.ascontiguousarray(p, float)
        d = np.ascontiguousarray(d, float)
        t = np.zeros(1)
        who = lib().or_hit(self.h, geom, _ptr(p), _ptr(d), float(ell), int(exclude), _ptr(t))
        return who, float(t[0])

    def collide(self, cath, v, V, u_b, u_psi):
        v = np.ascontiguousarray(v, float)
        V = np.ascontiguousarray(V, float)
        vo, Vo, chi = np.zeros(3), np.zeros(3), np.zeros(1)
        lib().or_collide(self.h, cath, _ptr(v), _ptr(V), float(u_b), float(u_psi), _ptr(vo), _ptr(Vo), _ptr(chi))
        return vo, Vo, float(chi[0])

    def partner(self, inst, pid, event, v, seed=None):
        v = np.ascontiguousarray(v, float)
        V = np.zeros(3)
        seed = self.scene.seed if seed is None else seed
        a = lib().or_partner(self.h, int(seed), inst, int(pid), int(event), _ptr(v), _ptr(V))
        return V, a

    def thermalize(self, inst, pid, E0, n_coll, seed=None):
        out = np.zeros(n_coll)
        seed = self.scene.seed if seed is None else seed
        lib().or_thermalize(self.h, int(seed), inst, int(pid), float(E0), int(n_coll), _ptr(out))
        return out

    def trace(self, inst, pid, rows=64, seed=None):
        out = np.zeros(rows * 10)
        seed = self.scene.seed if seed is None else seed
        lib().or_trace(self.h, int(seed), int(inst), int(pid), int(rows), _ptr(out))
        return out.reshape(rows, 10)

    def table_launch(self, cath, u_mu, u_E):
        """(mu, E) drawn from cathode cath's joint launch table for uniforms (u_mu, u_E)."""
        mu, E = C.c_double(), C.c_double()
        lib().or_table_launch(self.h, int(cath), float(u_mu), float(u_E), C.byref(mu), C.byref(E))
        return mu.value, E.value

    def plant_unweighted_partner(self, on=True):
        """Tests only: plant a known mistake (partner drawn from the plain Maxwellian)."""
        lib().or_scene_plant_unweighted_partner(self.h, 1 if on else 0)

    def set_at_cutoff(self, on):
        """Launch at E = E_max in launch() and the runs that follow (boundary runs)."""
        lib().or_scene_set_at_cutoff(self.h, 1 if on else 0)

    def launch(self, inst, pid, seed=None):
        p, d, E = np.zeros(3), np.zeros(3), np.zeros(1)
        seed = self.scene.seed if seed is None else seed
        lib().or_launch(self.h, int(seed), inst, int(pid), _ptr(p), _ptr(d), _ptr(E))
        return p, d, float(E[0])


# ------------------------------------------------------------- scalar probes
def chi(eps, beta, screening="moliere"):
    return lib().or_chi(0 if screening == "moliere" else 1, float(eps), float(beta))


def x0(eps, beta, screening="moliere"):
    return lib().or_x0(0 if screening == "moliere" else 1, float(eps), float(beta))


def chi_hard_sphere(beta):
    return lib().or_chi_hard_sphere(float(beta))


def bmax_direct(eps, chi_min, screening="moliere"):
    return lib().or_bmax_direct(0 if screening == "moliere" else 1, float(chi_min), float(eps))


def bmax_interp(eps, chi_min):
    return lib().or_bmax_interp(float(chi_min), float(eps))


def emax(k, M_i, M_t, E_i, U_s):
    return lib().or_emax(k, M_i, M_t, E_i, U_s)


def racetrack_cdf(r0, sigma, R, r):
    return lib().or_racetrack_cdf(r0, sigma, R, r)


def racetrack_r(r0, sigma, R, u):
    return lib().or_racetrack_r(r0, sigma, R, u)


def thompson(E_max, U, u):
    return lib().or_thompson(E_max, U, u)


def cos_mu(coef, u):
    c = np.ascontiguousarray(coef, float)
    return lib().or_cos_mu(_ptr(c), float(u))


def c_energy():
    return lib().or_c_energy()


def rel_speed_pdf(g, v, s):
    return lib().or_rel_speed_pdf(g, v, s)


def integrate_test(which, a, b):
    return lib().or_integrate_test(which, a, b)


def uniform_from_word(x):
    """RN in ]0,1] from a 32-bit Philox word (same mapping as the transporter)."""
    x = np.asarray(x, dtype=np.uint64)
    return ((x >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * 2.0 ** -24


# ------------------------------------------------------------------ tallies
def tally(scene, out):
    """Tallies from per-particle outcomes (instance-major layouts)."""
    g = scene.grid
    n_inst = len(scene.instances)
    ncell = g["nx"] * g["ny"]
    inst = out["inst"].astype(np.int64)
    prim = out["prim"].astype(np.int64)
    cell = out["cell"].astype(np.int64)
    max_prims = max(gg["prim_count"] for gg in scene.geometries)
    on_grid = cell >= 0
    counts = np.bincount(inst[on_grid] * ncell + cell[on_grid], minlength=n_inst * ncell).reshape(n_inst, ncell)
    energy = np.bincount(inst[on_grid] * ncell + cell[on_grid], weights=out["E"][on_grid],
                         minlength=n_inst * ncell).reshape(n_inst, ncell)
    landed = prim >= 0
    prim_counts = np.bincount(inst[landed] * max_prims + prim[landed],
                              minlength=n_inst * max_prims).reshape(n_inst, max_prims)
    timed_out = np.bincount(inst[~landed], minlength=n_inst)
    res = {"counts": counts, "energy": energy, "prim_counts": prim_counts, "timed_out": timed_out}
    if g["n_ebins"] > 0:
        eb = np.floor(out["E"][on_grid] / g["e_hist_max"] * g["n_ebins"]).astype(np.int64)
        eb = np.clip(eb, 0, g["n_ebins"] - 1)
        res["hist_E"] = np.bincount(inst[on_grid] * g["n_ebins"] + eb,
                                    minlength=n_inst * g["n_ebins"]).reshape(n_inst, -1)
    if g["n_abins"] > 0:
        theta = np.degrees(np.arccos(np.clip(out["cos"][on_grid], 0.0, 1.0)))
        ab = np.clip(np.floor(theta / 90.0 * g["n_abins"]).astype(np.int64), 0, g["n_abins"] - 1)
        res["hist_A"] = np.bincount(inst[on_grid] * g["n_abins"] + ab,
                                    minlength=n_inst * g["n_abins"]).reshape(n_inst, -1)
    return res


# ---------------------------------------------------------------- composition
def rate_line(points, power):
    """Sputter rate at `power` on the line through two (power, rate) points
    (linear power-rate relation of Fig. 4a / Table S1); returns (rate, slope)."""
    (p1, r1), (p2, r2) = points
    slope = (r2 - r1) / (p2 - p1)
    return r1 + slope * (power - p1), slope


def composition(counts, patch_of_cell, ref, rates, density, mass):
    """Arrival counts -> at.% (Methods paragraph after Table 1): the arrival
    fraction of element j at point m relative to the reference point, weighted
    with the sputter rate, then with bulk density / atomic mass, normalised.
    counts: [n_cath][n_cells]; returns comp [n_points][n_cath] and N [n_cath][n_points]."""
    counts = np.asarray(counts, dtype=np.float64)
    n_points = int(np.max(patch_of_cell)) + 1
    n_cath = counts.shape[0]
    N = np.zeros((n_cath, n_points))
    for j in range(n_cath):
        sel = patch_of_cell >= 0
        N[j] = np.bincount(patch_of_cell[sel], weights=counts[j][sel], minlength=n_points)
    a = np.empty((n_points, n_cath))
    for j in range(n_cath):
        a[:, j] = rates[j] * N[j] / N[j, ref] * density[j] / mass[j]
    return 100.0 * a / a.sum(axis=1, keepdims=True), N


def lr_gradient(outcomes, n_inst, n_cells, grad_counts):
    """Likelihood-ratio estimate of dL/d ln p per instance from per-particle
    scores: sum over landing particles of dL/dcount[cell] * score."""
    g = np.zeros(n_inst)
    on = outcomes["cell"] >= 0
    gc = np.asarray(grad_counts).reshape(n_inst, n_cells)
    np.add.at(g, outcomes["inst"][on], gc[outcomes["inst"][on], outcomes["cell"][on]] * outcomes["score"][on])
    return g
