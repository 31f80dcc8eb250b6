"""The measured peaks that the roofline divides by (sput_microbench, through the
C ABI) lie where the GB300's unit counts put them: 128 FP32 FMA lanes and 16
MUFU lanes per SM and clock (32 for ex2), at an SM clock no higher than the device's
maximum; the L2 reductions complete at a positive rate.  A peak far above its
unit-count ceiling would mean the timed kernel did not do its work."""

import pytest

pytestmark = pytest.mark.gpu


def test_peaks_within_unit_count_bounds():
    import torch

    from paper_2411_14413_gb300 import api

    assert torch.cuda.is_available()
    dev = torch.device("cuda", 0)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    clk_hz = 2.07e9  # maximum SM clock of the GB300 (nvidia-smi clocks.max.sm)
    scratch = torch.zeros(8 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    ffma = api.sput_microbench(0, "ffma", scratch, 4000, stream)
    assert ffma.ops_per_s <= 1.02 * n_sm * 128 * clk_hz, ffma.ops_per_s
    assert ffma.ops_per_s >= 0.5 * n_sm * 128 * clk_hz, ffma.ops_per_s
    # MUFU lanes per SM and clock: 16, and 32 for ex2 (measured at twice the others' rate)
    for kind, lanes in (("mufu_lg2", 16), ("mufu_ex2", 32), ("mufu_rsqrt", 16), ("mufu_sin", 16)):
        r = api.sput_microbench(0, kind, scratch, 2000, stream)
        assert 0.3 * n_sm * lanes * clk_hz <= r.ops_per_s <= 1.02 * n_sm * lanes * clk_hz, (kind, r.ops_per_s)
    ph = api.sput_microbench(0, "philox", scratch, 500, stream)
    # a block is at least 40 multiplies and 20 three-input xors (the key schedule can be
    # hoisted): at most the lane-issue ceiling / 60
    assert 0 < ph.ops_per_s <= n_sm * 128 * clk_hz / 60, ph.ops_per_s
    for kind in ("red_i32", "red_i64", "red_f64"):
        r = api.sput_microbench(0, kind, scratch, 500, stream, n_slots=160_000)
        assert r.ops_per_s > 1e9 and r.ops == r.blocks * r.threads * 500, (kind, r.ops_per_s)
