"""bench.py's pure helpers, on the CPU: the replica manifest of the batched
configuration, the SplitMix64 seeds, the launch counts and the roofline
arithmetic that the bench line reports."""
import sys

import numpy as np
import pytest

import bench


def test_splitmix64_first_outputs_from_state_zero():
    # the generator's published sequence (Steele, Lea, Flood 2014; Vigna's
    # splitmix64.c): state 0, then state + 0x9E3779B97F4A7C15
    assert bench.splitmix64(0) == 0xE220A8397B1DCDAF
    assert bench.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_batched_manifest_is_deterministic_and_in_range():
    L1, b1, s1 = bench.batched_replicas()
    L2, b2, s2 = bench.batched_replicas()
    np.testing.assert_array_equal(L1, L2)
    np.testing.assert_array_equal(b1, b2)          # exact doubles
    np.testing.assert_array_equal(s1, s2)
    assert len(L1) == 512
    assert set(np.unique(L1)) <= {32, 64, 128, 256, 512, 1024, 2048}
    T = 1.0 / b1
    assert T.min() >= 1.5 and T.max() <= 3.5
    assert len(set(s1.tolist())) == 512
    assert s1[0] == bench.splitmix64(11 << 32)
    # E[L^2] over the 7 sides is 798,866; the 512-replica sample is near it
    assert abs(float(np.mean(L1.astype(np.float64) ** 2)) / 798866.0 - 1.0) < 0.15


def test_batch_launch_count():
    # 4 lanes x 2 half-sweeps per sweep + one counter kernel per 50-sweep graph
    assert bench.batch_launches(512, 5000) == 2 * 5000 * 4 + 100
    assert bench.batch_launches(3, 10) == 2 * 10 * 3 + 1


def test_cluster_launch_count():
    # L = 296: pitch 8 words, 256-sweep pieces; 2280 records of 10 sweeps in
    # chunks of 1024, 1024 and 232 records: 40, 40 and 10 pieces
    assert bench.cluster_launches(296, 22800, 10) == (2 * 40 + 1) * 2 + 2 * 10 + 1
    # L = 512: pitch 14 words, 256-sweep pieces; one chunk of 20 records
    assert bench.cluster_launches(512, 200, 10) == 2 * 1 + 1
    assert bench.cluster_launches(512, 205, 10) == 2 * 1 + 1 + 2 * 1 + 1     # 5 sweeps after the last record
    # L = 1008: pitch 24 words, 256-sweep pieces (346 fit two 128 MB buffers)
    assert bench.cluster_launches(1008, 1960, 10) == 2 * 8 + 1
    # L = 2016: pitch 48 words, 86-sweep pieces (two 128 MB buffers)
    assert bench.cluster_launches(2016, 1960, 10) == 2 * 23 + 1


def test_two_pipe_roofline_arithmetic():
    peaks = {"sm_count": 152, "mulwide_per_sm_clk": 32.0, "mad32_per_sm_clk": 64.0, "lop3_per_sm_clk": 64.0,
             "sm_max_mhz": 2070.0, "clock_source": "test"}
    r = bench.two_pipe_roofline(1376.0, 10, peaks)
    # FMA-heavy only 8, ALU only 7.6, either 2: balanced 8.8 slots per pipe
    assert r["slots_per_site_per_pipe"] == pytest.approx(8.8)
    assert r["peak_spin_updates_per_ns"] == pytest.approx(152 * 64 * 2070e6 / 8.8 / 1e9)
    assert r["frac"] == pytest.approx(1376.0 / r["peak_spin_updates_per_ns"])
    r7 = bench.two_pipe_roofline(1.0, 7, peaks)
    assert r7["slots_per_site_per_pipe"] == pytest.approx((5.0 + 6.1 + 2.0) / 2)
    # a device whose wide product ran at the 32-bit rate: FMA-heavy only 4
    # slots, so the ALU-only work (7.6) binds
    r_fast = bench.two_pipe_roofline(1.0, 10, dict(peaks, mulwide_per_sm_clk=64.0))
    assert r_fast["slots_per_site_per_pipe"] == pytest.approx(7.6)


def test_default_arguments(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.steps, a.warmup, a.workload, a.impl, a.rng) == (1, 400, 5, "large", "gb300", 10)
    assert a.warmup >= 3
