"""sput_run_noalloc: the transport without any device allocation.

Callers that may not allocate device memory while they run (a global-mode
stream capture, a process whose device memory belongs to another allocator,
an allocation-free serving loop) use this entry point; it keeps its run
scratch in a static array of the library instead of a per-scene buffer.  The
test calls it through the C ABI twice in a row and compares each result with
the regular sput_run on the same scene, seed and tallies layout: integer
tallies bit-for-bit, FP64 energy sums to 1e-12 relative (atomic order).
This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process.
"""

import pytest

import workloads

pytestmark = pytest.mark.gpu


def _tallies(torch, layout, dev):
    from paper_2411_14413_gb300 import _native as N

    ni = layout.n_instances
    t = {
        "counts": torch.zeros((ni, layout.ny, layout.nx), dtype=torch.int64, device=dev),
        "energy": torch.zeros((ni, layout.ny, layout.nx), dtype=torch.float64, device=dev),
        "prim_counts": torch.zeros((ni, layout.max_prims), dtype=torch.int64, device=dev),
        "timed_out": torch.zeros((ni,), dtype=torch.int64, device=dev),
    }
    s = N.sput_tallies()
    for k, v in t.items():
        setattr(s, k, v.data_ptr())
    return t, s


def test_noalloc_matches_sput_run_twice():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import paper_2411_14413_gb300 as pkg
    from paper_2411_14413_gb300 import api

    pkg.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    sc = workloads.scene_quaternary(n_per_cathode=30000)
    h = api.sput_scene_create(sc, 0)
    try:
        lay = api.sput_tally_layout_get(h)
        stream = torch.cuda.current_stream(dev).cuda_stream
        ref, ref_s = _tallies(torch, lay, dev)
        st_ref = api.sput_run(h, api.run_opts(seed=11), stream, ref_s)
        for call in range(2):
            got, got_s = _tallies(torch, lay, dev)
            # leave garbage in the outputs first: the call must clear them itself
            got["counts"].fill_(7)
            got["energy"].fill_(3.0)
            st = api.sput_run_noalloc(h, api.run_opts(seed=11), stream, got_s)
            torch.cuda.synchronize(dev)
            for k in ("counts", "prim_counts", "timed_out"):
                assert torch.equal(ref[k], got[k]), (call, k)
            rel = (got["energy"] - ref["energy"]).abs().max() / ref["energy"].abs().max()
            assert float(rel) < 1e-12, (call, float(rel))
            assert st.particles == st_ref.particles == sc.total_particles
            assert st.collisions == st_ref.collisions and st.attempts == st_ref.attempts
    finally:
        api.sput_scene_destroy(h)
