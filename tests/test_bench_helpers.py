"""Host logic of bench.py: roofline arithmetic, the ncu counter record's
matching rules, and the serving pool's frame windows (no GPU needed)."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PROBE = {"fp64_fma_per_s": 5.0e11, "fp32_fma_per_s": 4.0e13}


def test_counter_record_matches_only_its_kernel_and_launch(monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "fit_kernel_counters.json")))
    launch = tuple(rec["launch"])
    c, note = bench.profiled_counters(rec["n_clusters"], launch)
    if rec["kernel_sha256_16"] != bench.kernel_source_hash():
        assert c is None and "changed" in note
        return
    assert c["dram_bytes"] == rec["dram_bytes_per_launch"] and "this launch" in note
    half, _ = bench.profiled_counters(rec["n_clusters"] // 2, launch)
    assert abs(half["warp_inst"] - rec["warp_inst_per_launch"] / 2) < 1.0
    other, why = bench.profiled_counters(rec["n_clusters"], (launch[0] * 2, launch[1]))
    assert other is None and "launch shape" in why
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    stale, why = bench.profiled_counters(rec["n_clusters"], launch)
    assert stale is None and "changed" in why


def test_roofline_fractions(monkeypatch):
    monkeypatch.setattr(bench, "profiled_counters", lambda n, l, v="": (
        {"dram_bytes": 64.0 * n, "warp_inst": 40.0 * n, "thread_inst": 40.0 * 28 * n, "fp32_flop_per_cluster": 700.0},
        "test"))
    nc, nt, t = 1_000_000, 10_000, 1e-3
    r = bench.fit_roofline(nc, nt, nc, t, (304, 256), PROBE, 152, 2000.0)
    # the binding roof: FP64 lane-operations against the live FP64 FMA rate
    assert r["bound"] == "alu" and r["binding"] == "fp64" and r["peak"] == pytest.approx(5.0e11 / 1e12)
    assert r["achieved"] == pytest.approx(bench.FP64_PER_CLUSTER * nc / t / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["frac_of_nominal"] == pytest.approx(bench.FP64_PER_CLUSTER * nc / t / bench.FP64_NOMINAL_OPS)
    side = r["beside"]
    assert side["fp32"]["frac"] == pytest.approx(700.0 * nc / t / 8.0e13)
    peaks, _ = bench.measured_peaks()
    assert side["hbm"]["frac"] == pytest.approx((22 * nc + 108 * nt) / t / 1e9 / peaks["hbm_gbs"])
    assert side["issue"]["peak_ginst_s"] == pytest.approx(4 * 152 * 2000e6 / 1e9)
    assert side["issue"]["frac"] == pytest.approx(40.0 * nc / t / (4 * 152 * 2000e6))
    assert r["traffic"] == 64.0 * nc and side["issue"]["active_lanes_per_inst"] == pytest.approx(28)


def test_roofline_without_counters_keeps_the_fp64_roof(monkeypatch):
    monkeypatch.setattr(bench, "profiled_counters", lambda n, l, v="": (None, "no record"))
    r = bench.fit_roofline(1000, 10, 1000, 1e-6, (1, 1), PROBE, 152, None)
    assert "FP64" in r["unit"] and r["traffic"] is None and r["frac"] == pytest.approx(11 * 1000 / 1e-6 / 5e11)
    assert "issue" not in r["beside"] and "fp32" not in r["beside"]


def test_serving_pool_windows():
    big, wins = bench.serving_pool(0, 12, pool_tracks=60_000, seed=3)
    off = big.offsets
    want = np.minimum(bench.tpcgen.lognormal_sizes(12, bench.SERVE_MEDIAN, bench.SERVE_SIGMA, bench.SERVE_LO,
                                                   bench.SERVE_HI, seed=3 + 77), off[-1] - 1)
    for (t0, t1), c in zip(wins, want):
        assert 0 <= t0 < t1 <= big.n_tracks
        got = off[t1] - off[t0]
        # the window holds the wanted clusters, up to one track, unless the pool ran out
        assert got >= min(c, off[-1] - off[t0]) and got - c < 400
    assert bench.percentile([1.0, 2.0, 3.0, 4.0], 50) == pytest.approx(2.5)


def test_ranks_take_their_frames_from_the_replica_shards():
    """Under torchrun each rank fits one independent frame, dealt round robin
    by the replica helpers: distinct seeds, every rank one frame."""
    for ws in (1, 2, 4, 8):
        seeds = [bench.frame_seed(r, ws) for r in range(ws)]
        assert sorted(seeds) == list(range(ws))
    assert bench.reduce_max(None, None, 3.5) == 3.5 and bench.reduce_sum(None, None, 2.0) == 2.0
