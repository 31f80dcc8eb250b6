"""Failure paths of the transport library, exercised without any GPU fault.

* timeout: a run with statistics and timeout_ms = 1 returns SPUT_ERR_TIMEOUT
  while its kernel is still running; the kernel then finishes normally and the
  tallies are complete and bit-identical to a run that was waited for.
* non-finite state: SPUT_RUN_INJECT_NONFINITE starts particle 0 of every
  instance with a NaN speed; the kernel retires it as timed out, sets the
  non-finite bit of device_status, and the call returns SPUT_ERR_DEVICE_CHECK;
  every other particle's record is unchanged.
* checked build: libsput_checked.so (every table, cell, primitive and record
  index tested against its buffer) gives bit-identical integer tallies and a
  clean status word on the single-Ni and quaternary scenes.
"""

import ctypes as C

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def pkg():
    import paper_2411_14413_gb300 as p
    p.build()
    return p


def test_timeout_returns_status_and_run_completes(torch, pkg):
    from paper_2411_14413_gb300 import _native as N
    from paper_2411_14413_gb300 import api

    sc = workloads.scene_quaternary(n_per_cathode=2_000_000)
    tr = pkg.Transport(sc)
    stream = torch.cuda.current_stream().cuda_stream
    ref = tr.run(seed=4)
    want = {k: v.clone() for k, v in tr.t.items()}
    with pytest.raises(N.SputError) as ei:
        api.sput_run(tr.h, api.run_opts(seed=4, timeout_ms=1), stream, tr._tal, True)
    assert ei.value.status == 4, ei.value          # SPUT_ERR_TIMEOUT
    torch.cuda.synchronize()                        # the kernel was left running and ends normally
    for k in ("counts", "prim_counts", "timed_out"):
        assert torch.equal(want[k], tr.t[k]), k
    assert int(tr.t["prim_counts"].sum() + tr.t["timed_out"].sum()) == sc.total_particles
    # the scene stays usable
    st = tr.run(seed=4)
    assert st.collisions == ref.collisions
    tr.close()


def test_nonfinite_injection_sets_status_bit(torch, pkg):
    from paper_2411_14413_gb300 import _native as N
    from paper_2411_14413_gb300 import api

    sc = workloads.scene_quaternary(n_per_cathode=5000)
    tr = pkg.Transport(sc, records=True)
    tr.run(seed=2)
    base = tr.records()
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(N.SputError) as ei:
        api.sput_run(tr.h, api.run_opts(seed=2, flags=N.SPUT_RUN_INJECT_NONFINITE), stream, tr._tal, True)
    assert ei.value.status == 5, ei.value          # SPUT_ERR_DEVICE_CHECK
    torch.cuda.synchronize()
    got = tr.records()
    first = np.arange(4) * 5000                     # particle 0 of each instance
    assert np.all(got["prim"][first] == -1)
    assert int(tr.t["timed_out"].sum()) == 4 + int(np.sum(base["prim"] == -1))
    others = np.setdiff1d(np.arange(sc.total_particles), first)
    assert np.array_equal(got["prim"][others], base["prim"][others])
    assert np.array_equal(got["cell"][others], base["cell"][others])
    # the status bit is reported in the statistics too
    st = N.sput_run_stats()
    rc = N.load().sput_run(tr.h, C.byref(api.run_opts(seed=2, flags=N.SPUT_RUN_INJECT_NONFINITE)),
                           C.c_void_p(stream), C.byref(tr._tal), C.byref(st))
    assert rc == 5 and (st.device_status & 1) == 1 and st.particles == sc.total_particles
    # a normal run afterwards is clean
    assert tr.run(seed=2).device_status == 0
    tr.close()


def _run_with(lib, torch, scene, seed):
    """Transport `scene` through the library handle `lib`; integer tallies and stats."""
    from paper_2411_14413_gb300 import _native as N
    from paper_2411_14413_gb300 import api

    d, keep = api.scene_desc(scene)
    h = C.c_void_p()
    N.check(lib.sput_scene_create(C.byref(d), 0, C.byref(h)), "sput_scene_create")
    lay = N.sput_tally_layout()
    N.check(lib.sput_tally_layout_get(h, C.byref(lay)), "layout")
    cdt = torch.int64 if lay.count_type == 1 else torch.int32
    t = {"counts": torch.zeros((lay.n_instances, lay.ny, lay.nx), dtype=cdt, device="cuda"),
         "prim_counts": torch.zeros((lay.n_instances, lay.max_prims), dtype=torch.int64, device="cuda"),
         "timed_out": torch.zeros((lay.n_instances,), dtype=torch.int64, device="cuda")}
    tal = N.sput_tallies()
    for k, v in t.items():
        setattr(tal, k, v.data_ptr())
    st = N.sput_run_stats()
    rc = lib.sput_run(h, C.byref(api.run_opts(seed=seed)), C.c_void_p(torch.cuda.current_stream().cuda_stream),
                      C.byref(tal), C.byref(st))
    torch.cuda.synchronize()
    lib.sput_scene_destroy(h)
    return rc, st, t


@pytest.mark.parametrize("name", ["single_ni", "quaternary"])
def test_checked_build_matches_regular(torch, pkg, name):
    from paper_2411_14413_gb300 import _native as N

    checked = N.load(path=N.CHECKED_LIB_PATH)
    regular = N.load()
    sc = workloads.scene_single_ni(n=100_000) if name == "single_ni" else workloads.scene_quaternary(n_per_cathode=100_000)
    rc_r, st_r, t_r = _run_with(regular, torch, sc, 9)
    rc_c, st_c, t_c = _run_with(checked, torch, sc, 9)
    assert rc_r == 0 and rc_c == 0, (rc_r, rc_c, checked.sput_last_error())
    assert st_c.device_status == 0
    for k in t_r:
        assert torch.equal(t_r[k], t_c[k]), k
    assert st_c.collisions == st_r.collisions and st_c.attempts == st_r.attempts
