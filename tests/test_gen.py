"""Synthetic frame generator: structure, determinism and distributions."""
import numpy as np
import pytest

import tpcgen


def test_structure_and_geometry():
    f = tpcgen.generate("detector50k", n_tracks=3000, truth=True)
    n = np.diff(f.offsets)
    assert f.offsets[0] == 0 and np.all(n >= 10) and np.all(n <= tpcgen.N_ROWS)
    for t in range(0, f.n_tracks, 97):
        r = f.row[f.offsets[t]:f.offsets[t + 1]].astype(int)
        assert np.all(np.diff(r) > 0)
    rx = tpcgen.row_x_table()
    assert np.array_equal(f.x, rx[f.row])
    # sector frame: |y| within the sector edge, |z| within the drift length
    assert np.all(np.abs(f.truth[:, 0]) <= f.x * np.tan(np.radians(10)) + 1e-9)
    assert np.all(np.abs(f.truth[:, 1]) <= 250.0)
    assert np.all(f.sy2 == np.float32(0.01)) and np.all(f.sz2 == np.float32(0.01))
    assert f.sector.max() < 36


def test_deterministic_and_thread_independent():
    a = tpcgen.generate("detector50k", n_tracks=2000, threads=1, seed=7)
    b = tpcgen.generate("detector50k", n_tracks=2000, threads=8, seed=7)
    c = tpcgen.generate("detector50k", n_tracks=2000, threads=3, seed=8)
    for k in ("offsets", "x", "y", "z", "row", "sector"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    assert not np.array_equal(a.y[:100], c.y[:100])


def test_dropout_and_outlier_rates():
    f = tpcgen.generate("detector50k", n_tracks=20000, truth=True)
    # dropout: clusters missing inside the crossed-row span
    n = np.diff(f.offsets)
    first, last = f.row[f.offsets[:-1]].astype(int), f.row[f.offsets[1:] - 1].astype(int)
    span = last - first + 1
    inner_missing = (span - n).sum() / (span - 2).clip(min=1).sum()
    assert 0.04 < inner_missing < 0.06
    assert 0.008 < f.flags.mean() < 0.012
    # outliers displaced by up to 2 cm, inliers Gaussian with sigma 0.1
    d = f.y.astype(np.float64) - f.truth[:, 0]
    inl = f.flags == 0
    assert abs(d[inl].std() - 0.1) < 0.002
    assert np.abs(d[~inl]).max() <= 2.0 + 0.6


def test_pt_spectra():
    f = tpcgen.generate("sector1k", n_tracks=5000, truth=True)
    pt = 1 / np.abs(f.truth_vertex[:, 5])
    assert pt.min() >= 0.2 - 1e-12 and pt.max() <= 10 + 1e-12
    g = tpcgen.generate("pbpb2m", n_tracks=5000, truth=True)
    assert np.median(1 / np.abs(g.truth_vertex[:, 5])) > 0.2  # short/curling tracks were redrawn


def test_subset_rebases_offsets():
    f = tpcgen.generate("sector1k", n_tracks=100)
    s = f.subset(10, 20)
    assert s.offsets[0] == 0 and s.n_tracks == 10
    assert np.array_equal(s.y, f.y[f.offsets[10]:f.offsets[20]])


def test_lognormal_and_poisson():
    v = tpcgen.lognormal_sizes(20000, 800, 1.0, 10, 20000, seed=0)
    assert v.min() >= 10 and v.max() <= 20000
    assert 700 < np.median(v) < 900
    t = tpcgen.poisson_arrivals(20000, 50.0, seed=0)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.02) < 0.001


def test_event_batch_shapes_and_independence():
    f, ev = tpcgen.event_batch(n_events=64, median=40, sigma_ln=1.0, lo=10, hi=400, seed=2)
    sizes = np.diff(ev)
    assert ev[0] == 0 and ev[-1] == f.n_tracks and sizes.min() >= 10 and sizes.max() <= 400
    assert 15 < np.median(sizes) < 110
    # an event equals the same tracks generated on their own (tracks keyed by index)
    e = 7
    t0, t1 = int(ev[e]), int(ev[e + 1])
    alone = tpcgen.generate("detector50k", seed=2, n_tracks=t1 - t0, track_id_offset=t0)
    sub = f.subset(t0, t1)
    assert np.array_equal(alone.offsets, sub.offsets)
    for k in ("x", "y", "z", "row"):
        assert np.array_equal(getattr(alone, k), getattr(sub, k)), k
