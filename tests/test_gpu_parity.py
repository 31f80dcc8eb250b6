"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP32 device arithmetic against FP64):
  * sub-steps: scattering angle within 2e-6 rad; b_max, K(v) and the partner
    envelope (A, B) within 2e-5 relative; launch position within 2e-4 mm, direction within 2e-5,
    energy within 2e-5 relative;
  * whole trajectories: at least 99.9 % of particles land on the same
    primitive and substrate cell as the oracle's (same Philox words drive
    both sides; the rest are decision flips at cell edges or acceptance
    thresholds), the others pass a chi-square two-sample test;
  * integers: sum of all landings + timed-out = N exactly; results are
    bit-identical across launch shapes and ticket chunking.
"""

import math

import numpy as np
import pytest
from scipy import stats

import workloads

pytestmark = pytest.mark.gpu

CHI_MIN = math.radians(1.0)


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


def _cell_parity(gpu, orc, min_frac=0.999):
    same = (gpu["prim"] == orc["prim"]) & (gpu["cell"] == orc["cell"])
    frac = float(same.mean())
    n = len(same)
    # allow the 0.1 % budget plus three binomial standard deviations of it
    allowed = (1 - min_frac) * n + 3 * math.sqrt((1 - min_frac) * n) + 1
    return frac, int((~same).sum()), allowed


# ----------------------------------------------------------------- sub-steps
def test_probe_chi_and_bmax(torch, pkg, oracle_mod):
    sc = workloads.scene_single_ni(n=10)
    tr = pkg.Transport(sc)
    # eps up to e^-3 covers every collision of these workloads (E_r < 700 eV for Ni-Ar)
    eps_list = np.exp(np.linspace(-27.0, -3.0, 25))
    x, ref = [], []
    for e in eps_list:
        bm = oracle_mod.bmax_interp(e, CHI_MIN)
        for ub in [0.0, 1e-6, 1e-3, 0.05, 0.2, 0.5, 0.8, 1.0]:
            b = bm * math.sqrt(ub)
            x += [e, b]
            ref.append(oracle_mod.chi(e, b))
    got = tr.probe("chi", 0, np.array(x))
    err = np.abs(got - np.array(ref))
    assert err.max() < 2e-6, (err.max(), np.argmax(err))
    bm_got = tr.probe("bmax", 0, eps_list)
    bm_ref = np.array([oracle_mod.bmax_interp(e, CHI_MIN) for e in eps_list])
    assert np.max(np.abs(bm_got / bm_ref - 1)) < 2e-5
    tr.close()


def test_probe_collision_deflection(torch, pkg, oracle_mod):
    """The deflection as a collision computes it from the impact-parameter uniform u
    (b = b_max sqrt(u)): the device's deflection table inside its range (ln eps in
    [-26, -4], ln(b/b_max) >= -6), the Gauss-Mehler integral outside, both against the
    oracle's adaptive quadrature at the oracle's own b_max."""
    sc = workloads.scene_single_ni(n=10)
    tr = pkg.Transport(sc)
    rng = np.random.default_rng(5)
    le = np.concatenate([rng.uniform(-27.0, -3.0, 3000), np.linspace(-26.0, -4.0, 45)])
    u = np.concatenate([rng.uniform(1e-7, 1.0, 3000), np.full(45, 1.0)])
    u[::7] = np.exp(2 * rng.uniform(-7.0, 0.0, len(u[::7])))      # deep into small b, below the table
    x = np.empty(2 * len(le))
    x[0::2], x[1::2] = np.exp(le), u
    got = tr.probe("chi_u", 0, x)
    ref = np.array([oracle_mod.chi(math.exp(a), oracle_mod.bmax_interp(math.exp(a), CHI_MIN) * math.sqrt(w))
                    for a, w in zip(le, u)])
    err = np.abs(got - ref)
    assert err.max() < 2e-6, (err.max(), le[err.argmax()], u[err.argmax()])
    inside = (le >= -26.0) & (le < -4.0) & (0.5 * np.log(u) >= -6.0)
    assert inside.sum() > 2000 and (~inside).sum() > 300
    tr.close()


@pytest.mark.parametrize("physics", [{}, {"interaction": "hard_sphere"}, {"gas_motion": "stationary"}])
def test_probe_rate_tables(torch, pkg, oracle_mod, physics):
    sc = workloads.scene_quaternary(n_per_cathode=10, physics=physics)
    tr = pkg.Transport(sc)
    o = oracle_mod.OracleScene(sc)
    for c in range(4):
        # speeds up to 200 eV of kinetic energy: inside every pair's table range
        m = sc.cathodes[c]["element"].mass
        v_hi = math.sqrt(2 * 200.0 / (m * oracle_mod.c_energy()))
        v = np.concatenate([[0.0, 1e-3], np.geomspace(0.01, v_hi, 40)])
        if physics.get("gas_motion") == "stationary":
            # at rest the Moliere sigma(v) diverges like ln^2(1/v) as v -> 0; the first
            # table pieces (v < 0.05 km/s, E < 1e-4 eV) are not meant to follow it
            v = v[v >= 0.05]
        K = tr.probe("K", c, v)
        Kr = np.array([o.K(c, x) for x in v])
        ok = Kr > 0
        assert np.max(np.abs(K[ok] / Kr[ok] - 1)) < 2e-5, (c, np.max(np.abs(K[ok] / Kr[ok] - 1)))
        if physics.get("gas_motion", "thermal") == "thermal":
            # the partner-rejection envelope (A, B) against the oracle's hull construction
            AB = tr.probe("M", c, v).reshape(-1, 2)
            ABr = np.array([o.envelope(c, x) for x in v])
            scale = ABr[:, 0] + 1.6 * ABr[:, 1]            # the envelope's size at the mean |V|/s
            assert np.max(np.abs(AB[:, 0] - ABr[:, 0]) / scale) < 2e-5, (c, np.abs(AB - ABr).max(0))
            assert np.max(np.abs(AB[:, 1] - ABr[:, 1]) / scale) < 2e-5, (c, np.abs(AB - ABr).max(0))
    tr.close()


def test_probe_launch(torch, pkg, oracle_mod):
    sc = workloads.scene_quaternary(n_per_cathode=60000)
    sc.cathodes[2]["cos_coef"] = (0.2, 0.5, 0.1, 0.0, 0.3, 0.05)   # exercise the general cosine sum
    tr = pkg.Transport(sc)
    o = oracle_mod.OracleScene(sc)
    for inst in range(4):
        # every 7th id plus the ids whose racetrack draw lies in either tail
        u = np.array([oracle_mod.uniform_from_word(oracle_mod.philox([pid, inst, 0, 0], [0, 0])[0])
                      for pid in range(20000)])
        tail = np.nonzero((u < 2e-3) | (u > 0.998))[0]
        assert len(tail) > 40
        pids = np.concatenate([np.arange(0, 4000, 7), tail]).astype(np.float64)
        got = tr.probe("launch", inst, pids)
        for j, pid in enumerate(pids):
            p, d, E = o.launch(inst, int(pid))
            assert np.max(np.abs(got[j, :3] - p)) < 2e-4, (inst, pid, got[j, :3], p)
            assert np.max(np.abs(got[j, 3:6] - d)) < 2e-5
            assert abs(got[j, 6] / E - 1) < 2e-5
    tr.close()


def test_trace_parity(torch, pkg, oracle_mod):
    """Flight-by-flight states of sampled particles follow the oracle's until
    the end (or until a decision flips, which must stay rare)."""
    sc = workloads.scene_single_ni(n=400)
    tr = pkg.Transport(sc)
    o = oracle_mod.OracleScene(sc)
    pids = np.arange(0, 400, 2)
    G = tr.probe("trace", 0, pids.astype(np.float64))
    diverged = 0
    max_dp = 0.0
    for j, pid in enumerate(pids):
        O = o.trace(0, int(pid))
        Gj = G[j]
        for r in range(Gj.shape[0]):
            if O[r, 7] == -2 and Gj[r, 7] == -2:
                break
            same_kind = Gj[r, 7] == O[r, 7] and (Gj[r, 7] == -1 or Gj[r, 8] == O[r, 8])
            if not same_kind:
                diverged += 1
                break
            max_dp = max(max_dp, float(np.max(np.abs(Gj[r, :3] - O[r, :3]))))
    assert diverged <= 2, diverged
    assert max_dp < 5e-3, max_dp
    tr.close()


# ------------------------------------------------------- whole trajectories
def _run_both(pkg, oracle_mod, sc, **kw):
    tr = pkg.Transport(sc, records=True, energy=True)
    st = tr.run(**kw)
    g = tr.records()
    tal = {k: v.cpu().numpy() for k, v in tr.t.items() if k != "records"}
    tr.close()
    o = oracle_mod.OracleScene(sc).run_all()
    return g, o, st, tal


@pytest.mark.parametrize("name,n", [("single_ni", 6000), ("quaternary", 1500)])
def test_trajectory_parity(torch, pkg, oracle_mod, name, n):
    sc = workloads.scene_by_name(name, **({"n": n} if name == "single_ni" else {"n_per_cathode": n}))
    g, o, st, tal = _run_both(pkg, oracle_mod, sc)
    N = sc.total_particles
    assert st.particles == N and st.landed + st.timed_out == N
    assert tal["prim_counts"].sum() + tal["timed_out"].sum() == N
    frac, bad, allowed = _cell_parity(g, o)
    assert bad <= allowed, (frac, bad, allowed)
    assert np.array_equal(g["ncoll"] == 0, o["ncoll"] == 0) or np.mean(g["ncoll"] == o["ncoll"]) > 0.99
    # arrival energies of matching particles agree to FP32 accuracy
    same = (g["prim"] == o["prim"]) & (g["ncoll"] == o["ncoll"])
    rel = np.abs(g["E"][same] / o["E"][same] - 1)
    assert np.median(rel) < 1e-5
    # GPU tallies are the sums of its own records
    counts = tal["counts"].reshape(len(sc.instances), -1)
    inst = np.repeat(np.arange(len(sc.instances)), [i["n"] for i in sc.instances])
    on = g["cell"] >= 0
    want = np.bincount(inst[on] * counts.shape[1] + g["cell"][on], minlength=counts.size).reshape(counts.shape)
    assert np.array_equal(counts, want)


def test_tally_chi_square_against_oracle(torch, pkg, oracle_mod):
    """Landing distributions over primitives agree in a two-sample chi-square test."""
    sc = workloads.scene_single_ni(n=6000)
    g, o, st, tal = _run_both(pkg, oracle_mod, sc)
    a = np.bincount(g["prim"] + 1, minlength=10)
    b = np.bincount(o["prim"] + 1, minlength=10)
    keep = (a + b) > 0
    chi2, p, _, _ = stats.chi2_contingency(np.vstack([a[keep], b[keep]]))
    assert p > 0.01


@pytest.mark.parametrize("physics", [{"interaction": "hard_sphere"},
                                     {"interaction": "hard_sphere", "gas_motion": "stationary", "max_collisions": 150},
                                     {"max_collisions": 3}])
def test_trajectory_parity_test_modes(torch, pkg, oracle_mod, physics):
    sc = workloads.scene_single_ni(n=3000, physics=physics)
    g, o, st, tal = _run_both(pkg, oracle_mod, sc)
    frac, bad, allowed = _cell_parity(g, o)
    assert bad <= allowed, (frac, bad, allowed)
    assert tal["prim_counts"].sum() + tal["timed_out"].sum() == 3000


def test_vacuum_parity_exact(torch, pkg, oracle_mod):
    """p = 0: straight flights only; every particle lands where the oracle's does."""
    sc = workloads.scene_single_ni(n=20000, pressure=0.0)
    g, o, st, tal = _run_both(pkg, oracle_mod, sc)
    assert st.collisions == 0
    frac, bad, allowed = _cell_parity(g, o, min_frac=0.9995)
    assert bad <= allowed, (frac, bad)


# ------------------------------------------------------------- determinism
def test_bit_exact_across_launch_shapes_and_chunks(torch, pkg):
    sc = workloads.scene_quaternary(n_per_cathode=20000)
    tr = pkg.Transport(sc, energy=False)
    tr.run(block_threads=128, ticket_chunk=32)
    ref = {k: v.clone() for k, v in tr.t.items()}
    for bt, ch, bps in [(64, 1, 0), (256, 128, 1), (96, 7, 2)]:
        tr.run(block_threads=bt, ticket_chunk=ch, blocks_per_sm=bps)
        for k in ref:
            assert torch.equal(ref[k], tr.t[k]), (k, bt, ch)
    # the same tickets in three chunks, accumulated
    n = sc.total_particles
    cuts = [0, n // 3, (2 * n) // 3 + 11, n]
    for i in range(3):
        tr.run(ticket_begin=cuts[i], ticket_end=cuts[i + 1], accumulate=i > 0)
    for k in ref:
        assert torch.equal(ref[k], tr.t[k]), k
    tr.close()


def test_edge_cases(torch, pkg):
    sc = workloads.scene_quaternary(n_per_cathode=5)
    sc.instances[1]["n"] = 0          # an empty instance between non-empty ones
    sc.instances[3]["n"] = 1
    tr = pkg.Transport(sc)
    st = tr.run()
    assert st.particles == 11
    assert int(tr.t["prim_counts"][1].sum()) == 0
    st = tr.run(ticket_begin=4, ticket_end=4)   # empty range
    assert st.particles == 0
    assert int(tr.t["counts"].sum()) == 0
    tr.close()


# ------------------------------------------------ full-size sampled parity
def test_full_size_quaternary_sampled_parity(torch, pkg, oracle_mod):
    """The 4 x 1e7 quaternary workload in the default launch shape; 4000
    sampled particles recomputed one by one by the oracle."""
    sc = workloads.scene_quaternary()
    tr = pkg.Transport(sc, records=True, energy=True)
    st = tr.run()
    N = sc.total_particles
    assert st.particles == N and st.landed + st.timed_out == N
    assert int(tr.t["prim_counts"].sum() + tr.t["timed_out"].sum()) == N
    rng = np.random.default_rng(2024)
    tick = np.sort(rng.choice(N, 4000, replace=False))
    rec = tr.t["records"][torch.from_numpy(tick).to(tr.t["records"].device)].cpu().numpy()
    tr.close()
    n_per = sc.instances[0]["n"]
    o = oracle_mod.OracleScene(sc).run_ids((tick // n_per).astype(np.int32), (tick % n_per).astype(np.uint64))
    g = {"prim": rec[:, 0], "cell": rec[:, 1]}
    frac, bad, allowed = _cell_parity(g, o)
    assert bad <= allowed, (frac, bad, allowed)


def test_rng_stream_common_random_numbers(torch, pkg, oracle_mod):
    """Instances on the same Philox stream (sput_instance.rng_stream) with the same
    conditions transport the same particle ids identically on the device, and the
    device follows the oracle with the streams set."""
    sc = workloads.scene_quaternary(n_per_cathode=2000)
    sc.instances[2] = dict(sc.instances[0], rng_stream=1)
    sc.instances[0] = dict(sc.instances[0], rng_stream=1)
    sc.instances[3] = dict(sc.instances[3], rng_stream=7)
    tr = pkg.Transport(sc, records=True)
    tr.run()
    g = tr.records()
    counts = tr.t["counts"].cpu().numpy()
    tr.close()
    a, c = slice(0, 2000), slice(4000, 6000)
    for k in ("prim", "cell", "ncoll"):
        assert np.array_equal(g[k][a], g[k][c]), k
    assert np.array_equal(counts[0], counts[2])
    o = oracle_mod.OracleScene(sc).run_all()
    frac, bad, allowed = _cell_parity(g, o)
    assert bad <= allowed, (frac, bad, allowed)
