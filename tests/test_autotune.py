"""Host logic of the autotuner: candidate space, selection, tune table."""
import json

import pytest

from paper_2402_01205_gb300 import autotune as A


def test_candidates_cover_every_shape_once():
    c = A.candidates()
    keys = {tuple(sorted(d.items())) for d in c}
    assert len(keys) == len(c) == 2 * (A.MAX_BLOCKS_PER_SM[128] + A.MAX_BLOCKS_PER_SM[256])
    assert all(1 <= d["blocks_per_sm"] <= A.MAX_BLOCKS_PER_SM[d["block_threads"]] for d in c)


def test_tune_picks_fastest_and_ties_go_first():
    cands = A.candidates(block_threads=(256,), sort_tracks=(1,))
    cands = cands + [{"block_threads": 256, "blocks_per_sm": 3, "sort_tracks": 1}]
    ms = {1: 30.0, 2: 12.5, 3: 12.5}
    e = A.tune(None, None, cands=cands, timer=lambda c: ms[c["blocks_per_sm"]])
    assert e["choice"] == {"block_threads": 256, "blocks_per_sm": 2, "sort_tracks": 1}
    assert e["ms"] == 12.5 and [r["ms"] for r in e["all"]] == [12.5, 12.5, 30.0]
    with pytest.raises(ValueError):
        A.select({})


def test_table_roundtrip_and_nearest_class(tmp_path):
    p = str(tmp_path / "tune.json")
    assert A.load(p) == {}
    e_small = {"choice": {"block_threads": 128, "blocks_per_sm": 6, "sort_tracks": 1}, "ms": 1.0}
    e_big = {"choice": {"block_threads": 256, "blocks_per_sm": 3, "sort_tracks": 1}, "ms": 9.0}
    A.save(p, A.table_key("GB300", 152, 5_000), e_small)
    A.save(p, A.table_key("GB300", 152, 5_000_000), e_big)
    t = A.load(p)
    assert json.load(open(p)) == t and len(t) == 2
    assert A.lookup(t, "GB300", 152, 4_000_000) == e_big          # same class
    assert A.lookup(t, "GB300", 152, 8_000) == e_small            # nearest class
    assert A.lookup(t, "B200", 148, 8_000) is None                 # other device
    assert A.config_for(e_big) == {"block_threads": 256, "blocks_per_sm": 3, "sort_tracks": 1}
    assert A.config_for(None) == {}
    assert A.size_class(0) == "nt4^0" and A.size_class(4 ** 5) == "nt4^5"
