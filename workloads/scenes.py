"""Synthetic sputter-system scenes (chamber, dummy objects, cathodes, conditions).

A scene mirrors the object model the paper describes for a sputter system
(Sec. "The SIMTRA Python wrapper"): a vacuum chamber with gas, temperature and
pressure; one or more magnetrons, each with an element, a racetrack and a
3D body; and "dummy" objects (substrate, holder, shields) that collect every
atom that reaches them.  Coordinates are millimetres; the chamber is an
axis-aligned box whose six walls absorb.

Primitive kinds (all surfaces absorb on both faces):
  box       the chamber interior (the only kind that is hit from inside)
  rect      planar rectangle: centre, in-plane unit axes u, v, half sizes p0, p1
  disc      planar disc or annulus: centre, in-plane axes u, v, radii p0 (inner), p1 (outer)
  cylinder  open tube: centre, unit axis u, radius p0, half length p1
The plane normal of rect/disc is u x v.

Nothing here samples, transports or tallies; it only places objects and fixes
process conditions, so that the CUDA path and the oracle read identical
inputs.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .elements import ELEMENTS, GAS_AR, Element

INCH_MM = 25.4


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


@dataclass
class Scene:
    name: str
    box_lo: tuple
    box_hi: tuple
    gas: Element
    T: float                       # K
    prims: List[dict]
    geometries: List[dict]         # {"prim_begin", "prim_count", "substrate"} (substrate: local index)
    cathodes: List[dict]
    instances: List[dict]          # {"geometry", "cathode", "pressure" (Pa), "E_i" (eV), "k", "n"}
    grid: dict
    physics: dict = field(default_factory=dict)
    seed: int = 0

    @property
    def total_particles(self) -> int:
        return int(sum(int(i["n"]) for i in self.instances))

    def with_particles(self, n) -> "Scene":
        """Copy with every instance's particle count set to n (int or list)."""
        import copy
        s = copy.deepcopy(self)
        ns = n if isinstance(n, (list, tuple, np.ndarray)) else [n] * len(s.instances)
        for inst, k in zip(s.instances, ns):
            inst["n"] = int(k)
        return s

    def with_physics(self, **kw) -> "Scene":
        import copy
        s = copy.deepcopy(self)
        s.physics.update(kw)
        return s

    def with_ion_energy(self, E_i) -> "Scene":
        """Copy with the incident ion energy (eV) of every instance set (scalar or list)."""
        import copy
        s = copy.deepcopy(self)
        es = E_i if isinstance(E_i, (list, tuple, np.ndarray)) else [E_i] * len(s.instances)
        for inst, e in zip(s.instances, es):
            inst["E_i"] = float(e)
        return s

    def with_pressure(self, p) -> "Scene":
        import copy
        s = copy.deepcopy(self)
        ps = p if isinstance(p, (list, tuple, np.ndarray)) else [p] * len(s.instances)
        for inst, q in zip(s.instances, ps):
            inst["pressure"] = float(q)
        return s


def default_physics(**kw) -> dict:
    phys = {
        "chi_min_deg": 1.0,          # CM-angle cut-off that defines the total cross section
        "interaction": "moliere",    # "moliere" | "hard_sphere"
        "hs_diameter": 3.0,          # Angstrom, only for the hard-sphere test potential
        "gas_motion": "thermal",     # "thermal" | "stationary"
        "max_attempts": 32,          # partner rejection attempts per collision
        "max_collisions": 1_000_000, # per particle; beyond it the particle is counted as timed out
        "thermal_switch_eV": 0.0,    # diffusion shortcut for thermalised atoms below this energy (0 = off)
    }
    phys.update(kw)
    return phys


def default_grid(nx, ny, half_u, half_v, count_dtype="int64", energy=True,
                 n_ebins=0, e_hist_max=160.0, n_abins=0) -> dict:
    return {
        "nx": int(nx), "ny": int(ny), "half_u": float(half_u), "half_v": float(half_v),
        "count_dtype": count_dtype, "energy": bool(energy),
        "n_ebins": int(n_ebins), "e_hist_max": float(e_hist_max), "n_abins": int(n_abins),
    }


def _prim(kind, center=(0, 0, 0), u=(1, 0, 0), v=(0, 1, 0), p0=0.0, p1=0.0):
    return {
        "kind": kind,
        "center": tuple(float(x) for x in center),
        "u": tuple(float(x) for x in u),
        "v": tuple(float(x) for x in v),
        "p0": float(p0),
        "p1": float(p1),
    }


def cathode_pose(azimuth_deg: float, tilt_deg: float, radial_mm: float, z_mm: float):
    """Target-surface centre, outward normal and in-plane reference axis of a
    cathode whose axis is tilted by `tilt_deg` towards the chamber axis."""
    ph = math.radians(azimuth_deg)
    ta = math.radians(tilt_deg)
    c = np.array([radial_mm * math.cos(ph), radial_mm * math.sin(ph), z_mm])
    n = np.array([-math.sin(ta) * math.cos(ph), -math.sin(ta) * math.sin(ph), math.cos(ta)])
    e1 = np.array([math.cos(ta) * math.cos(ph), math.cos(ta) * math.sin(ph), math.sin(ta)])
    return c, _unit(n), _unit(e1)


def cathode_assembly(c, n, e1, target_radius=INCH_MM, chimney_radius=30.0,
                     chimney_top=10.0, body_depth=40.0):
    """Target disc, chimney tube and back plate of one magnetron (3 primitives).

    The target disc faces the chamber (normal n); the chimney is a tube of
    radius `chimney_radius` from `body_depth` behind the target surface to
    `chimney_top` in front of it; the back plate closes the tube."""
    c = np.asarray(c, float)
    n = _unit(n)
    e1 = _unit(e1)
    e2 = np.cross(n, e1)
    target = _prim("disc", c, e1, e2, 0.0, target_radius)
    mid = 0.5 * (chimney_top - body_depth)
    chimney = _prim("cylinder", c + mid * n, n, e1, chimney_radius, 0.5 * (chimney_top + body_depth))
    back = _prim("disc", c - body_depth * n, e1, -e2, 0.0, chimney_radius)
    return [target, chimney, back]


def _cathode(el: Element, c, n, e1, target_local, r0=12.0, sigma=3.0, R=INCH_MM,
             cos_coef=(0, 1, 0, 0, 0, 0)):
    return {
        "element": el,
        "center": tuple(float(x) for x in c),
        "normal": tuple(float(x) for x in n),
        "e1": tuple(float(x) for x in e1),
        "racetrack": {"kind": "gaussian_annulus", "r0": float(r0), "sigma": float(sigma), "R": float(R)},
        "cos_coef": tuple(float(x) for x in cos_coef),
        "target": int(target_local),
    }


def _substrate_group(center_z, substrate_kind, box_top, half=50.0):
    """Substrate (facing -z), holder plate behind it and the holder shaft."""
    u = (1.0, 0.0, 0.0)
    v = (0.0, -1.0, 0.0)       # u x v = -z: the front face looks down at the cathodes
    if substrate_kind == "rect":
        sub = _prim("rect", (0, 0, center_z), u, v, half, half)
    else:
        sub = _prim("disc", (0, 0, center_z), u, v, 0.0, half)
    holder = _prim("disc", (0, 0, center_z + 1.0), u, v, 0.0, 70.0)
    z0 = center_z + 1.0
    shaft = _prim("cylinder", (0, 0, 0.5 * (z0 + box_top)), (0, 0, 1), (1, 0, 0), 10.0, 0.5 * (box_top - z0))
    return [sub, holder, shaft]


# ---------------------------------------------------------------------------
# Single Ni cathode: 2-inch target, Gaussian annulus racetrack r0=12 sigma=3 mm,
# Ar 0.5 Pa 300 K, E_i = 400 eV, U_s = 4.44 eV, cosine emission, 1e5 particles,
# 400x400x300 mm box, 100x100 mm substrate at 100 mm, 50x50 int32 tally.
# ---------------------------------------------------------------------------
def scene_single_ni(n=100_000, pressure=0.5, E_i=400.0, T=300.0, nx=50, ny=50,
                    count_dtype="int32", energy=False, physics=None, seed=0) -> Scene:
    box_lo, box_hi = (-200.0, -200.0, -100.0), (200.0, 200.0, 200.0)
    c, nrm, e1 = cathode_pose(0.0, 0.0, 0.0, 0.0)
    prims = [_prim("box")]
    prims += cathode_assembly(c, nrm, e1)
    sub_local = len(prims)
    prims += _substrate_group(100.0, "rect", box_hi[2])
    geoms = [{"prim_begin": 0, "prim_count": len(prims), "substrate": sub_local}]
    cath = [_cathode(ELEMENTS["Ni"], c, nrm, e1, target_local=1)]
    inst = [{"geometry": 0, "cathode": 0, "pressure": float(pressure), "E_i": float(E_i), "k": 0.4, "n": int(n)}]
    grid = default_grid(nx, ny, 50.0, 50.0, count_dtype=count_dtype, energy=energy)
    return Scene("single_ni", box_lo, box_hi, GAS_AR, float(T), prims, geoms, cath, inst, grid,
                 default_physics(**(physics or {})), seed)


# ---------------------------------------------------------------------------
# Joint (polar cosine, energy) launch table standing in for the binned output
# of a binary-collision code for the target: an energy spectrum peaking at a few
# eV with a power-law tail, whose angular distribution narrows towards the
# normal as the energy grows (exponent 0.6 at low E, towards 2 at high E).
# ---------------------------------------------------------------------------
def synthetic_launch_table(n_mu=32, n_E=64, E_hi=150.0, E_peak=3.0) -> dict:
    mu = (np.arange(n_mu) + 0.5) / n_mu
    E = (np.arange(n_E) + 0.5) * E_hi / n_E
    expo = 0.6 + 1.4 * E / (E + 20.0)
    w = mu[:, None] ** expo[None, :] * (E / (E + 2.0 * E_peak) ** 2.5)[None, :]
    return {"weights": w, "E_hi": float(E_hi)}


def scene_single_ni_table(n=100_000, table=None, **kw) -> Scene:
    """The single-Ni scene with its cathode launching from a joint (mu, E) table."""
    import copy
    sc = copy.deepcopy(scene_single_ni(n=n, **kw))
    sc.cathodes[0]["launch_table"] = table if table is not None else synthetic_launch_table()
    sc.name = "single_ni_table"
    return sc


# ---------------------------------------------------------------------------
# Quaternary co-sputter Ni/Pd/Pt/Ru: cathodes at azimuth 0/90/180/270 deg,
# tilted 30 deg, axes meeting at the substrate centre 120 mm from each target;
# 100 mm wafer, 200x200 int64 counts + fp64 energy per cathode.
# ---------------------------------------------------------------------------
QUATERNARY = ("Ni", "Pd", "Pt", "Ru")


def _quaternary_geometry(tilt_deg, focus_z=100.0, throw=120.0, radial=None, z=None,
                         box_hi_z=200.0):
    prims = [_prim("box")]
    poses = []
    for i, _ in enumerate(QUATERNARY):
        az = 90.0 * i
        if radial is None:
            # confocal: target centre = focus - throw * normal
            ta = math.radians(tilt_deg)
            rad = throw * math.sin(ta)
            zc = focus_z - throw * math.cos(ta)
        else:
            rad, zc = radial, z
        c, nrm, e1 = cathode_pose(az, tilt_deg, rad, zc)
        poses.append((c, nrm, e1, len(prims)))
        prims += cathode_assembly(c, nrm, e1)
    sub_local = len(prims)
    prims += _substrate_group(focus_z, "disc", box_hi_z)
    return prims, poses, sub_local


def scene_quaternary(n_per_cathode=10_000_000, pressure=0.5, E_i=400.0, T=300.0, tilt_deg=30.0,
                     nx=200, ny=200, physics=None, seed=0, elements=QUATERNARY) -> Scene:
    box_lo, box_hi = (-200.0, -200.0, -100.0), (200.0, 200.0, 200.0)
    prims, poses, sub_local = _quaternary_geometry(tilt_deg, box_hi_z=box_hi[2])
    geoms = [{"prim_begin": 0, "prim_count": len(prims), "substrate": sub_local}]
    cath, inst = [], []
    for i, sym in enumerate(elements):
        c, nrm, e1, tloc = poses[QUATERNARY.index(sym)]
        cath.append(_cathode(ELEMENTS[sym], c, nrm, e1, target_local=tloc))
        inst.append({"geometry": 0, "cathode": i, "pressure": float(pressure), "E_i": float(E_i),
                     "k": 0.4, "n": int(n_per_cathode)})
    grid = default_grid(nx, ny, 50.0, 50.0, count_dtype="int64", energy=True)
    return Scene("quaternary", box_lo, box_hi, GAS_AR, float(T), prims, geoms, cath, inst, grid,
                 default_physics(**(physics or {})), seed)


# ---------------------------------------------------------------------------
# Batched sweep: 4 cathodes x 16 pressures (0.2-2 Pa, log) x 8 tilts (0-40 deg);
# per-instance particle counts uniform integers in [1e5, 1e7] (seed 0);
# 100x100 int64 tally per instance.  The target centres stay where the 30 deg
# confocal layout puts them; the tilt turns each cathode towards the axis.
# ---------------------------------------------------------------------------
def scene_tilt_pressure_sweep(n_range=(100_000, 10_000_000), n_pressures=16, n_tilts=8,
                              p_range=(0.2, 2.0), tilt_range=(0.0, 40.0), T=300.0, E_i=400.0,
                              nx=100, ny=100, physics=None, seed=0, counts_seed=0) -> Scene:
    box_lo, box_hi = (-200.0, -200.0, -100.0), (200.0, 200.0, 200.0)
    ta30 = math.radians(30.0)
    radial, zc = 120.0 * math.sin(ta30), 100.0 - 120.0 * math.cos(ta30)
    pressures = np.geomspace(p_range[0], p_range[1], n_pressures)
    tilts = np.linspace(tilt_range[0], tilt_range[1], n_tilts)
    prims, geoms, cath = [], [], []
    for t in tilts:
        gprims, poses, sub_local = _quaternary_geometry(float(t), radial=radial, z=zc, box_hi_z=box_hi[2])
        geoms.append({"prim_begin": len(prims), "prim_count": len(gprims), "substrate": sub_local})
        for i, sym in enumerate(QUATERNARY):
            c, nrm, e1, tloc = poses[i]
            cath.append(_cathode(ELEMENTS[sym], c, nrm, e1, target_local=tloc))
        prims += gprims
    rng = np.random.default_rng(counts_seed)
    n_inst = len(QUATERNARY) * n_pressures * n_tilts
    counts = rng.integers(n_range[0], n_range[1] + 1, size=n_inst)
    inst = []
    j = 0
    for ti in range(n_tilts):
        for pi in range(n_pressures):
            for ci in range(len(QUATERNARY)):
                inst.append({"geometry": ti, "cathode": ti * len(QUATERNARY) + ci,
                             "pressure": float(pressures[pi]), "E_i": float(E_i), "k": 0.4,
                             "n": int(counts[j])})
                j += 1
    grid = default_grid(nx, ny, 50.0, 50.0, count_dtype="int64", energy=False)
    return Scene("sweep", box_lo, box_hi, GAS_AR, float(T), prims, geoms, cath, inst, grid,
                 default_physics(**(physics or {})), seed)


# ---------------------------------------------------------------------------
# Tilt scan: one materials library (a subset of Ni/Pd/Pt/Ru, e.g. the ternary
# Pd-Pt-Ru library) simulated at several common cathode tilts in one launch.
# Target centres stay at the 30 deg confocal positions, as in the sweep; the
# instances are tilt-major (tilt t, element j -> instance t * n_el + j), so the
# count tallies of one tilt are contiguous; 200x200 int64 counts per instance.
# ---------------------------------------------------------------------------
def scene_tilt_scan(tilts, elements=("Pd", "Pt", "Ru"), n_per_cathode=1_000_000, pressure=0.5, T=300.0,
                    E_i=400.0, nx=200, ny=200, physics=None, seed=0, common_random_numbers=False) -> Scene:
    """One library at several common tilts, tilt-major (len(elements) instances per tilt).
    With common_random_numbers every tilt's instance of an element draws that element's
    random stream (the same particle ids and random numbers at every tilt)."""
    box_lo, box_hi = (-200.0, -200.0, -100.0), (200.0, 200.0, 200.0)
    ta30 = math.radians(30.0)
    radial, zc = 120.0 * math.sin(ta30), 100.0 - 120.0 * math.cos(ta30)
    prims, geoms, cath, inst = [], [], [], []
    for ti, t in enumerate(tilts):
        gprims, poses, sub_local = _quaternary_geometry(float(t), radial=radial, z=zc, box_hi_z=box_hi[2])
        geoms.append({"prim_begin": len(prims), "prim_count": len(gprims), "substrate": sub_local})
        for sym in elements:
            c, nrm, e1, tloc = poses[QUATERNARY.index(sym)]
            cath.append(_cathode(ELEMENTS[sym], c, nrm, e1, target_local=tloc))
            inst.append({"geometry": ti, "cathode": len(cath) - 1, "pressure": float(pressure), "E_i": float(E_i),
                         "k": 0.4, "n": int(n_per_cathode)})
            if common_random_numbers:
                inst[-1]["rng_stream"] = elements.index(sym) + 1
        prims += gprims
    grid = default_grid(nx, ny, 50.0, 50.0, count_dtype="int64", energy=False)
    return Scene("tilt_scan", box_lo, box_hi, GAS_AR, float(T), prims, geoms, cath, inst, grid,
                 default_physics(**(physics or {})), seed)


# ---------------------------------------------------------------------------
# Large: single Ni cathode, Ar 3 Pa, 1e9 particles, 64 primitives (chimney,
# substrate group and 57 seeded shields placed off the cathode-substrate line
# of sight), 512x512 grid + 64-bin energy + 32-bin arrival-angle histograms.
# ---------------------------------------------------------------------------
def scene_large_shielded(n=1_000_000_000, pressure=3.0, E_i=400.0, T=300.0, nx=512, ny=512,
                         physics=None, seed=0, shields_seed=0) -> Scene:
    box_lo, box_hi = (-200.0, -200.0, -100.0), (200.0, 200.0, 200.0)
    c, nrm, e1 = cathode_pose(0.0, 0.0, 0.0, 0.0)
    prims = [_prim("box")]
    prims += cathode_assembly(c, nrm, e1)
    sub_local = len(prims)
    prims += _substrate_group(100.0, "rect", box_hi[2])
    rng = np.random.default_rng(shields_seed)
    # 16 vertical planar baffles near the side walls
    for i in range(16):
        ang = 2 * math.pi * (i + rng.uniform(0.1, 0.9)) / 16
        rad = rng.uniform(150.0, 185.0)
        ctr = (rad * math.cos(ang), rad * math.sin(ang), rng.uniform(-40.0, 150.0))
        tang = (-math.sin(ang), math.cos(ang), 0.0)
        prims.append(_prim("rect", ctr, tang, (0, 0, 1), rng.uniform(10.0, 25.0), rng.uniform(15.0, 40.0)))
    # 16 horizontal annular rings at large radius
    for i in range(16):
        zr = -80.0 + i * (270.0 / 16) + rng.uniform(0.0, 5.0)
        r_in = rng.uniform(120.0, 150.0)
        prims.append(_prim("disc", (0, 0, zr), (1, 0, 0), (0, 1, 0), r_in, rng.uniform(r_in + 20.0, 195.0)))
    # 8 vertical posts
    for i in range(8):
        ang = 2 * math.pi * (i + 0.5) / 8
        rad = rng.uniform(100.0, 170.0)
        prims.append(_prim("cylinder", (rad * math.cos(ang), rad * math.sin(ang), 50.0), (0, 0, 1), (1, 0, 0),
                           rng.uniform(4.0, 9.0), rng.uniform(40.0, 120.0)))
    # 17 small clips around the substrate, outside its footprint
    for i in range(17):
        ang = 2 * math.pi * (i + rng.uniform(0.2, 0.8)) / 17
        rad = rng.uniform(85.0, 110.0)
        ctr = (rad * math.cos(ang), rad * math.sin(ang), rng.uniform(95.0, 110.0))
        prims.append(_prim("rect", ctr, (math.cos(ang), math.sin(ang), 0.0), (0, 0, 1),
                           rng.uniform(3.0, 8.0), rng.uniform(2.0, 6.0)))
    assert len(prims) == 64, len(prims)
    geoms = [{"prim_begin": 0, "prim_count": len(prims), "substrate": sub_local}]
    cath = [_cathode(ELEMENTS["Ni"], c, nrm, e1, target_local=1)]
    inst = [{"geometry": 0, "cathode": 0, "pressure": float(pressure), "E_i": float(E_i), "k": 0.4, "n": int(n)}]
    grid = default_grid(nx, ny, 50.0, 50.0, count_dtype="int64", energy=True,
                        n_ebins=64, e_hist_max=160.0, n_abins=32)
    return Scene("large", box_lo, box_hi, GAS_AR, float(T), prims, geoms, cath, inst, grid,
                 default_physics(**(physics or {})), seed)


_BUILDERS = {
    "single_ni": scene_single_ni,
    "single_ni_table": scene_single_ni_table,
    "quaternary": scene_quaternary,
    "sweep": scene_tilt_pressure_sweep,
    "tilt_scan": scene_tilt_scan,
    "large": scene_large_shielded,
}


def scene_by_name(name: str, **kw) -> Scene:
    return _BUILDERS[name](**kw)
