"""Thin Python binding of libsput.so.

The functions mirror the C entry points of ``include/sput.h`` one to one and
only marshal arguments: scene descriptions from ``workloads.Scene`` into the
ABI structs, torch tensors into device pointers, numpy arrays into host
pointers.  Every step of the transport runs in the CUDA library.  PyTorch
provides device memory and streams only.
"""

from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _native as N


def _lib():
    return N.load()


# ----------------------------------------------------------- marshalling
def scene_desc(scene):
    """Build the sput_scene_desc (and keep the arrays it points to alive)."""
    keep = []
    prims = (N.sput_primitive * len(scene.prims))()
    for i, P in enumerate(scene.prims):
        q = prims[i]
        q.kind = N.PRIM_KIND[P["kind"]]
        q.center[:] = P["center"]
        q.u[:] = P["u"]
        q.v[:] = P["v"]
        q.p0, q.p1 = P["p0"], P["p1"]
    geoms = (N.sput_geometry * len(scene.geometries))()
    for i, g in enumerate(scene.geometries):
        geoms[i].prim_begin, geoms[i].prim_count, geoms[i].substrate = g["prim_begin"], g["prim_count"], g["substrate"]
    cath = (N.sput_cathode * len(scene.cathodes))()
    for i, c in enumerate(scene.cathodes):
        q = cath[i]
        el = c["element"]
        rt = c["racetrack"]
        if rt["kind"] != "gaussian_annulus":
            raise ValueError("only the Gaussian-annulus racetrack is supported")
        q.Z, q.mass, q.U_s, q.target = el.Z, el.mass, el.U_s, c["target"]
        q.center[:] = c["center"]
        q.normal[:] = c["normal"]
        q.e1[:] = c["e1"]
        q.rt_r0, q.rt_sigma, q.rt_R = rt["r0"], rt["sigma"], rt["R"]
        q.cos_coef[:] = c["cos_coef"]
        lt = c.get("launch_table")
        if lt is not None:
            w = np.ascontiguousarray(lt["weights"], dtype=np.float64)
            if w.ndim != 2:
                raise ValueError("launch_table weights must be a 2-D array [n_mu][n_E]")
            keep.append(w)
            q.launch_table = w.ctypes.data_as(C.POINTER(C.c_double))
            q.n_mu, q.n_E = w.shape
            q.E_hi = float(lt["E_hi"])
    inst = instance_array(scene)
    d = N.sput_scene_desc()
    d.abi_version = N.SPUT_ABI_VERSION
    d.n_prims, d.n_geoms, d.n_cathodes, d.n_instances = len(prims), len(geoms), len(cath), len(inst)
    d.chamber.box_lo[:] = scene.box_lo
    d.chamber.box_hi[:] = scene.box_hi
    d.chamber.gas_Z = scene.gas.Z
    d.chamber.gas_mass = scene.gas.mass
    d.chamber.gas_T = scene.T
    d.prims = C.cast(prims, C.POINTER(N.sput_primitive))
    d.geoms = C.cast(geoms, C.POINTER(N.sput_geometry))
    d.cathodes = C.cast(cath, C.POINTER(N.sput_cathode))
    d.instances = C.cast(inst, C.POINTER(N.sput_instance))
    g = scene.grid
    d.grid.nx, d.grid.ny, d.grid.half_u, d.grid.half_v = g["nx"], g["ny"], g["half_u"], g["half_v"]
    d.grid.count_type = N.COUNT_TYPE[g["count_dtype"]]
    d.grid.n_ebins, d.grid.e_hist_max, d.grid.n_abins = g["n_ebins"], g["e_hist_max"], g["n_abins"]
    ph = scene.physics
    d.physics.chi_min = math.radians(ph["chi_min_deg"])
    d.physics.hs_diameter = ph["hs_diameter"]
    d.physics.interaction = N.INTERACTION[ph["interaction"]]
    d.physics.gas_motion = N.GAS_MOTION[ph["gas_motion"]]
    d.physics.max_attempts = ph["max_attempts"]
    d.physics.max_collisions = ph["max_collisions"]
    d.physics.thermal_switch_eV = float(ph.get("thermal_switch_eV", 0.0))
    return d, (prims, geoms, cath, inst, keep)


def instance_array(scene):
    inst = (N.sput_instance * len(scene.instances))()
    for i, I in enumerate(scene.instances):
        q = inst[i]
        q.geometry, q.cathode = I["geometry"], I["cathode"]
        q.pressure, q.E_i, q.k, q.n_particles = I["pressure"], I["E_i"], I["k"], int(I["n"])
        q.rng_stream = int(I.get("rng_stream", 0))
    return inst


# ------------------------------------------------ entry points (same names)
def sput_version():
    return _lib().sput_version()


def sput_scene_create(scene, device=0):
    d, keep = scene_desc(scene)
    h = C.c_void_p()
    N.check(_lib().sput_scene_create(C.byref(d), int(device), C.byref(h)), "sput_scene_create")
    return h


def sput_instances_set(handle, scene):
    inst = instance_array(scene)
    N.check(_lib().sput_instances_set(handle, inst, len(inst)), "sput_instances_set")


def sput_tally_layout_get(handle):
    lay = N.sput_tally_layout()
    N.check(_lib().sput_tally_layout_get(handle, C.byref(lay)), "sput_tally_layout_get")
    return lay


def sput_run(handle, opts, stream, tallies, want_stats=True):
    st = N.sput_run_stats()
    rc = _lib().sput_run(handle, C.byref(opts), C.c_void_p(stream), C.byref(tallies),
                         C.byref(st) if want_stats else None)
    N.check(rc, "sput_run")
    return st if want_stats else None


def sput_run_noalloc(handle, opts, stream, tallies, want_stats=True):
    """sput_run without any device allocation (static run scratch)."""
    st = N.sput_run_stats()
    rc = _lib().sput_run_noalloc(handle, C.byref(opts), C.c_void_p(stream), C.byref(tallies),
                                 C.byref(st) if want_stats else None)
    N.check(rc, "sput_run_noalloc")
    return st if want_stats else None


def sput_run_host(handle, opts, tallies):
    st = N.sput_run_stats()
    N.check(_lib().sput_run_host(handle, C.byref(opts), C.byref(tallies), C.byref(st)), "sput_run_host")
    return st


def sput_scene_destroy(handle):
    if handle:
        _lib().sput_scene_destroy(handle)


def sput_probe(handle, what, idx, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = len(x) // 2 if what in ("chi", "chi_u") else len(x)
    width = {"launch": 7, "trace": N.TRACE_ROWS * 10, "M": 2}.get(what, 1)
    y = np.zeros(n * width, dtype=np.float64)
    rc = _lib().sput_probe(handle, N.PROBE[what], int(idx), int(n), x.ctypes.data_as(C.c_void_p),
                           y.ctypes.data_as(C.c_void_p))
    N.check(rc, "sput_probe")
    if what == "launch":
        return y.reshape(n, 7)
    if what == "trace":
        return y.reshape(n, N.TRACE_ROWS, 10)
    return y


def run_opts(seed=0, ticket_begin=0, ticket_end=0, accumulate=False, block_threads=0, blocks_per_sm=0,
             ticket_chunk=0, timeout_ms=0, flags=0):
    o = N.sput_run_opts()
    o.seed, o.ticket_begin, o.ticket_end = int(seed), int(ticket_begin), int(ticket_end)
    o.accumulate, o.block_threads, o.blocks_per_sm = int(bool(accumulate)), int(block_threads), int(blocks_per_sm)
    o.ticket_chunk, o.timeout_ms, o.flags = int(ticket_chunk), int(timeout_ms), int(flags)
    return o


def sput_autotune(handle, opts, stream, tallies, sample_tickets):
    res = N.sput_tune_result()
    rc = _lib().sput_autotune(handle, C.byref(opts), C.c_void_p(stream), C.byref(tallies), int(sample_tickets),
                              C.byref(res))
    N.check(rc, "sput_autotune")
    return res


def sput_graph_create(handle, opts, stream, tallies):
    g = C.c_void_p()
    N.check(_lib().sput_graph_create(handle, C.byref(opts), C.c_void_p(stream), C.byref(tallies), C.byref(g)),
            "sput_graph_create")
    return g


def sput_graph_launch(graph, seed, stream):
    N.check(_lib().sput_graph_launch(graph, int(seed), C.c_void_p(stream)), "sput_graph_launch")


def sput_graph_destroy(graph):
    if graph:
        _lib().sput_graph_destroy(graph)


def sput_microbench(device, kind, scratch, iters, stream, n_slots=0):
    """Throughput of one unit (see include/sput.h); scratch is a device tensor."""
    res = N.sput_microbench_result()
    k = N.MICROBENCH_KINDS[kind] if isinstance(kind, str) else int(kind)
    rc = _lib().sput_microbench(int(device), k, int(n_slots), C.c_void_p(scratch.data_ptr()),
                                scratch.numel() * scratch.element_size(), int(iters), C.c_void_p(stream), C.byref(res))
    N.check(rc, "sput_microbench")
    return res


# ------------------------------------------------------------ convenience
class Transport:
    """A scene resident on one GPU plus torch-allocated tallies.

    ``run()`` transports every particle (or a ticket range) and returns the
    device tallies; nothing is computed in Python."""

    def __init__(self, scene, device=0, energy=None, score=False, records=False, prim_counts=True, score_T=False,
                 histograms=None):
        import torch

        self.scene = scene
        self.device = device
        self.h = sput_scene_create(scene, device)
        self.layout = sput_tally_layout_get(self.h)
        L = self.layout
        dev = torch.device("cuda", device)
        ni, nc = L.n_instances, L.nx * L.ny
        cdt = torch.int64 if L.count_type == 1 else torch.int32
        self.t = {"counts": torch.zeros((ni, L.ny, L.nx), dtype=cdt, device=dev)}
        if energy if energy is not None else scene.grid.get("energy", False):
            self.t["energy"] = torch.zeros((ni, L.ny, L.nx), dtype=torch.float64, device=dev)
        if score:
            self.t["score"] = torch.zeros((ni, L.ny, L.nx), dtype=torch.float64, device=dev)
        if score_T:
            self.t["score_T"] = torch.zeros((ni, L.ny, L.nx), dtype=torch.float64, device=dev)
        if prim_counts:
            self.t["prim_counts"] = torch.zeros((ni, L.max_prims), dtype=torch.int64, device=dev)
            self.t["timed_out"] = torch.zeros((ni,), dtype=torch.int64, device=dev)
        hist = histograms if histograms is not None else True
        if hist and L.n_ebins > 0:
            self.t["hist_E"] = torch.zeros((ni, L.n_ebins), dtype=torch.int64, device=dev)
        if hist and L.n_abins > 0:
            self.t["hist_A"] = torch.zeros((ni, L.n_abins), dtype=torch.int64, device=dev)
        if records:
            self.t["records"] = torch.zeros((int(L.n_tickets), 6), dtype=torch.int32, device=dev)
        self._tal = N.sput_tallies()
        for k, v in self.t.items():
            setattr(self._tal, k, v.data_ptr())

    def close(self):
        if getattr(self, "h", None):
            sput_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_instances(self, scene):
        self.scene = scene
        sput_instances_set(self.h, scene)

    def run(self, seed=None, stream=None, want_stats=True, **kw):
        import torch

        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        o = run_opts(seed=self.scene.seed if seed is None else seed, **kw)
        return sput_run(self.h, o, s, self._tal, want_stats)

    def records(self):
        """Per-particle records as numpy structured fields (device -> host)."""
        r = self.t["records"].cpu().numpy()
        return {
            "prim": r[:, 0].copy(), "cell": r[:, 1].copy(), "E": r[:, 2].view(np.float32).astype(np.float64),
            "cos": r[:, 3].view(np.float32).astype(np.float64), "ncoll": r[:, 4].view(np.uint32).astype(np.int64),
            "score": r[:, 5].view(np.float32).astype(np.float64),
        }

    def probe(self, what, idx, x):
        return sput_probe(self.h, what, idx, x)

    def autotune(self, sample_tickets=20_000_000, stream=None, **kw):
        """Time candidate launch shapes on a sample and keep the fastest as this scene's default."""
        import torch

        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        return sput_autotune(self.h, run_opts(seed=self.scene.seed, **kw), s, self._tal, sample_tickets)

    def graph(self, stream=None, **kw):
        """CUDA graph of one run into this object's tallies; replay with graph_launch(g, seed)."""
        import torch

        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        return sput_graph_create(self.h, run_opts(seed=self.scene.seed, **kw), s, self._tal)
