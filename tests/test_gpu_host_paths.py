"""Host-buffer entry point and int32 tallies of the gradient kernels."""

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2411_14413_gb300 as p
    p.build()
    return p


def test_run_host_matches_device_run_with_every_tally(pkg):
    """sput_run_host (host buffers, staged and copied by the library) gives the
    device run's tallies, the temperature score included, and accumulates."""
    import torch
    from paper_2411_14413_gb300 import _native as N, api

    sc = workloads.scene_single_ni(n=50_000)
    tr = pkg.Transport(sc, energy=True, score=True, score_T=True)
    tr.run(seed=11)
    dev = {k: v.cpu().numpy() for k, v in tr.t.items()}
    host = {k: torch.zeros_like(v, device="cpu").pin_memory() for k, v in tr.t.items()}
    ht = N.sput_tallies()
    for k, v in host.items():
        setattr(ht, k, v.data_ptr())
    api.sput_run_host(tr.h, api.run_opts(seed=11), ht)
    for k in ("counts", "prim_counts", "timed_out"):
        assert np.array_equal(host[k].numpy(), dev[k]), k
    for k in ("energy", "score", "score_T"):
        assert np.allclose(host[k].numpy(), dev[k], rtol=1e-12, atol=1e-12), k
    api.sput_run_host(tr.h, api.run_opts(seed=11, accumulate=True), ht)
    assert np.array_equal(host["counts"].numpy(), 2 * dev["counts"])
    tr.close()


def test_emax_backward_int32_counts(pkg, oracle_mod):
    """sput_emax_backward on an int32-count scene against the same contraction in numpy."""
    import torch
    from paper_2411_14413_gb300 import _native as N

    sc = workloads.scene_single_ni(n=200_000)
    assert sc.grid["count_dtype"] == "int32"
    tr = pkg.Transport(sc)
    cut = pkg.Transport(sc)
    tr.run(seed=2)
    cut.run(seed=2, flags=N.SPUT_RUN_LAUNCH_AT_CUTOFF)
    rng = np.random.default_rng(0)
    g = torch.as_tensor(rng.normal(size=tr.t["counts"].shape), device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    N.check(N.load().sput_emax_backward(tr.h, g.data_ptr(), tr.t["counts"].data_ptr(), cut.t["counts"].data_ptr(),
                                        out.data_ptr(), torch.cuda.current_stream().cuda_stream), "sput_emax_backward")
    o = oracle_mod.OracleScene(sc)
    Em, U = o.emax(0), sc.cathodes[0]["element"].U_s
    m_ar, m_ni = workloads.GAS_AR.mass, sc.cathodes[0]["element"].mass
    k_lambda = 0.4 * 4 * m_ar * m_ni / (m_ar + m_ni) ** 2
    diff = cut.t["counts"].cpu().numpy().astype(np.float64) - tr.t["counts"].cpu().numpy()
    want = k_lambda * 2 * U / (Em * (Em + U)) * float((g.cpu().numpy() * diff).sum())
    assert abs(out.item() - want) < 1e-5 * (abs(want) + 1e-9), (out.item(), want)
    tr.close()
    cut.close()
