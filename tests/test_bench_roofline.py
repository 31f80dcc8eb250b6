"""The bench line's roofline arithmetic (host code of bench.py).

The algorithmic work of a run is the method's own operations counted from the run's statistics
(flights F, partner attempts A, collisions C, particles N) and the geometry's primitive count P:
work = F (116 + 25 P) + 135 A + 78 C + 280 N lane-ops.  frac = work / kernel time / the measured
FP32 FMA lane-op rate; issue_frac uses the executed lane-instructions per collision instead.
The record below is one measured bench step of the quaternary workload (4 x 1e7 atoms, 16
primitives, means over 5 timed steps); its frac and issue_frac must come out by hand."""

import pytest

import bench
import workloads

# one measured bench record: per-step statistics, mean kernel time (ms), FMA peak (lane-ops/s)
RECORD = {"particles": 40_000_000, "flights": 971_285_517.4, "collisions": 931_285_517.4,
          "attempts": 1.2277208482658188 * 931_285_517.4}
KERNEL_MS = 71.75290222167969
FFMA = 39_163_256_736_553.51
EXEC_PER_COLLISION = 1891.0


def test_work_model_per_unit():
    assert bench.WORK_MODEL == {"philox_block": 100, "flight": 116, "prim_test": 25, "partner_attempt": 135,
                                "collision": 78, "particle": 280}
    one = {"particles": 0, "flights": 1, "collisions": 0, "attempts": 0}
    assert bench.algorithmic_lane_ops(one, 16) == 116 + 25 * 16
    assert bench.algorithmic_lane_ops({**one, "flights": 0, "attempts": 1}, 16) == 135
    assert bench.algorithmic_lane_ops({**one, "flights": 0, "collisions": 1}, 16) == 78
    assert bench.algorithmic_lane_ops({**one, "flights": 0, "particles": 1}, 16) == 280


def test_primitives_per_flight():
    assert bench.mean_prims(workloads.scene_quaternary(n_per_cathode=10)) == 16
    sc = workloads.scene_large_shielded(n=10)
    assert bench.mean_prims(sc) == 64


def test_frac_reproduces_the_measured_record_by_hand():
    work = (RECORD["flights"] * (116 + 25 * 16) + RECORD["attempts"] * 135 + RECORD["collisions"] * 78
            + RECORD["particles"] * 280)
    frac_by_hand = work / (KERNEL_MS / 1e3) / FFMA
    issue_by_hand = EXEC_PER_COLLISION * RECORD["collisions"] / (KERNEL_MS / 1e3) / FFMA
    e = bench.roofline_entry([RECORD], [KERNEL_MS], 16, {"ffma": FFMA}, EXEC_PER_COLLISION)
    assert e["frac"] == pytest.approx(frac_by_hand, rel=1e-12)
    assert e["issue_frac"] == pytest.approx(issue_by_hand, rel=1e-12)
    # the values that record printed in its line
    assert e["frac"] == pytest.approx(0.26311625172337416, rel=1e-9)
    assert e["issue_frac"] == pytest.approx(0.6266948221629213, rel=1e-9)
    assert e["algorithmic_lane_ops_per_collision"] == pytest.approx(793.93, abs=0.01)
    assert e["bound"] == "alu" and e["unit"] == "Tlane-op/s"
    assert e["achieved"] / e["peak"] == pytest.approx(e["frac"], rel=1e-12)
