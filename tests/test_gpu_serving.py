"""Serving through the C-ABI: resident slots, HBM-budget admission, overlap,
and results identical alone and in the mix."""
import time
import types

import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_01205_gb300 as T
    from paper_2402_01205_gb300 import _build
    _build.build()
    return T


def pinned_frame(f):
    g = types.SimpleNamespace()
    for k in ("offsets", "x", "y", "z", "sy2", "sz2", "row"):
        a = torch.from_numpy(np.ascontiguousarray(getattr(f, k)))
        setattr(g, k, a.pin_memory())
    return g


def frames_of_uneven_size(seed=0):
    pool = tpcgen.generate("detector50k", n_tracks=60_000, seed=seed)
    sizes = [800, 25_000, 3_000, 12_000, 150, 9_000]
    out, t0 = [], 0
    for s in sizes:
        out.append(pool.subset(t0, t0 + s))
        t0 += s
    return out


def alone(T, f):
    with T.Fitter() as fx:
        return fx.fit(f)


def test_results_identical_alone_and_in_the_mix(T):
    frames = frames_of_uneven_size()
    ref = [alone(T, f) for f in frames]
    with T.Fitter(max_slots=3) as fx:
        res = [T.alloc_result(f.n_tracks, f.n_clusters, pinned=True) for f in frames]
        tickets = [fx.submit(pinned_frame(f), r) for f, r in zip(frames, res)]
        for tk in tickets:
            st, t_done = fx.wait(tk, timeout_s=60)
            assert st == T.DONE and t_done > 0
    for r, rf in zip(res, ref):
        for k in rf:
            assert np.array_equal(r[k].numpy(), rf[k], equal_nan=k in ('state', 'cov')), k


def test_budget_admission_and_rejection(T):
    frames = frames_of_uneven_size(seed=1)
    big = max(frames, key=lambda f: f.n_clusters)
    # budget for about one large frame: frames are admitted one by one and all finish
    budget = int(big.n_clusters * 24 + big.n_tracks * 140 + (4 << 20))
    with T.Fitter(hbm_budget_bytes=budget, max_slots=4) as fx:
        res = [T.alloc_result(f.n_tracks, f.n_clusters, pinned=True) for f in frames]
        tickets = [fx.submit(pinned_frame(f), r) for f, r in zip(frames, res)]
        states = [fx.wait(tk, timeout_s=60)[0] for tk in tickets]
        assert states == [T.DONE] * len(frames)
        # a frame larger than the whole budget is refused at submission
        huge = tpcgen.generate("detector50k", n_tracks=40_000, seed=2)
        with pytest.raises(T.TpcfitError) as ei:
            fx.submit(pinned_frame(huge), T.alloc_result(huge.n_tracks, huge.n_clusters, pinned=True))
        assert ei.value.code == T.E_NOMEM
    for r, f in zip(res, frames):
        assert np.array_equal(r["status"].numpy(), alone(T, f)["status"])


def test_malformed_frame_rejected_neighbours_succeed(T):
    frames = frames_of_uneven_size(seed=3)[:3]
    bad = tpcgen.Frame(frames[1].offsets.copy(), *(getattr(frames[1], k) for k in ("x", "y", "z", "sy2", "sz2", "row")),
                       frames[1].sector)
    bad.offsets[5] = bad.offsets[7]
    with T.Fitter() as fx:
        r0 = T.alloc_result(frames[0].n_tracks, frames[0].n_clusters, pinned=True)
        t0 = fx.submit(pinned_frame(frames[0]), r0)
        with pytest.raises(T.TpcfitError) as ei:
            fx.submit(pinned_frame(bad), T.alloc_result(bad.n_tracks, bad.n_clusters, pinned=True))
        assert ei.value.code == T.E_INVAL
        r2 = T.alloc_result(frames[2].n_tracks, frames[2].n_clusters, pinned=True)
        t2 = fx.submit(pinned_frame(frames[2]), r2)
        assert fx.wait(t0, 60)[0] == T.DONE and fx.wait(t2, 60)[0] == T.DONE
        # a reported ticket is forgotten; unknown tickets are reported as such
        with pytest.raises(T.TpcfitError) as ei:
            fx.poll(t0)
        assert ei.value.code == T.E_NOTFOUND


def test_poll_pending_then_done_and_wait_timeout(T):
    f = tpcgen.generate("pbpb2m", n_tracks=300_000, seed=4)
    with T.Fitter() as fx:
        r = T.alloc_result(f.n_tracks, f.n_clusters, pinned=True)
        tk = fx.submit(pinned_frame(f), r)
        st, _ = fx.poll(tk)
        assert st in (T.PENDING, T.DONE)
        if st == T.PENDING:
            with pytest.raises(T.TpcfitError) as ei:
                fx.wait(tk, timeout_s=1e-6)
            assert ei.value.code in (T.E_TIMEOUT,)
        deadline = time.time() + 60
        while st == T.PENDING and time.time() < deadline:
            st, t_done = fx.poll(tk)
            time.sleep(0.001)
        assert st == T.DONE


def test_frame_split_into_parts_equals_plain_fit(T):
    """A served frame larger than host_chunk_clusters is fitted as several
    parts on several slots; the results are those of one plain fit."""
    f = tpcgen.generate("detector50k", n_tracks=20_000, seed=6)
    ref = alone(T, f)
    with T.Fitter(host_chunk_clusters=250_000, max_slots=3) as fx:  # about 9 parts, 3 slots
        res = [T.alloc_result(f.n_tracks, f.n_clusters, pinned=True) for _ in range(2)]
        tickets = [fx.submit(pinned_frame(f), r) for r in res]
        for t in tickets:
            assert fx.wait(t, 60)[0] == T.DONE
    for r in res:
        for k in ref:
            assert np.array_equal(ref[k], r[k].numpy(), equal_nan=k in ("state", "cov")), k


def test_served_fit_variant_equals_its_plain_fit(T):
    """Served frames (split into parts) use the handle's fit variant too."""
    f = tpcgen.generate("detector50k", n_tracks=8_000, seed=7)
    cfg = dict(xrho_per_row=0.01, fit_iterations=1)
    with T.Fitter(**cfg) as fx:
        ref = fx.fit(f)
    with T.Fitter(host_chunk_clusters=200_000, max_slots=3, **cfg) as fx:
        r = T.alloc_result(f.n_tracks, f.n_clusters, pinned=True)
        assert fx.wait(fx.submit(pinned_frame(f), r), 60)[0] == T.DONE
    for k in ref:
        assert np.array_equal(ref[k], r[k].numpy(), equal_nan=k in ("state", "cov")), k


def test_engine_fits_the_parts_of_several_frames_in_one_launch(T):
    """The serving engine fits every part that is ready in one persistent
    launch (warps take (part, group) descriptors from a device table): with
    many small frames submitted at once, launches fit several parts each, and
    every frame's results equal its plain fit, including residual codes."""
    pool = tpcgen.generate("detector50k", n_tracks=24_000, seed=11)
    frames = [pool.subset(i * 1_000, (i + 1) * 1_000 - 7 * i) for i in range(24)]
    ref = []
    with T.Fitter() as fx:
        for f in frames:
            r = T.alloc_result(f.n_tracks, f.n_clusters, residuals=True)
            fx.fit(f, r)
            ref.append(r)
    pinned = [pinned_frame(f) for f in frames]  # pinned first: the submissions follow one another at once
    with T.Fitter(max_slots=16) as fx:
        assert fx.serve_stats() == {"launches": 0, "parts": 0, "max_parts_per_launch": 0}
        res = [T.alloc_result(f.n_tracks, f.n_clusters, pinned=True, residuals=True) for f in frames]
        tickets = [fx.submit(p, r) for p, r in zip(pinned, res)]
        for tk in tickets:
            assert fx.wait(tk, timeout_s=60)[0] == T.DONE
        st = fx.serve_stats()
    assert st["parts"] == len(frames)
    assert st["launches"] < len(frames) and st["max_parts_per_launch"] >= 2, st
    for r, rf in zip(res, ref):
        for k in rf:
            assert np.array_equal(r[k].numpy(), rf[k], equal_nan=k in ("state", "cov")), k


def test_engine_under_budget_pressure_with_few_slots_and_small_parts(T):
    """Frames of random sizes (1 to 4,000 tracks) through 3 slots, parts of
    about 150,000 clusters and a budget of about two of the largest frames:
    admission waits for memory and slots, engine launches take whatever parts
    are ready, and every ticket finishes with the results of its plain fit."""
    pool = tpcgen.generate("detector50k", n_tracks=60_000, seed=21)
    sizes = np.random.default_rng(5).integers(1, 4_000, size=30)
    frames, t0 = [], 0
    for s in sizes:
        frames.append(pool.subset(t0, t0 + int(s)))
        t0 += int(s)
    ref = [alone(T, f) for f in frames]
    big = max(frames, key=lambda f: f.n_clusters)
    budget = int(2 * (big.n_clusters * 24 + big.n_tracks * 140) + (8 << 20))
    pinned = [pinned_frame(f) for f in frames]
    with T.Fitter(hbm_budget_bytes=budget, max_slots=3, host_chunk_clusters=150_000) as fx:
        res = [T.alloc_result(f.n_tracks, f.n_clusters, pinned=True) for f in frames]
        tickets = [fx.submit(p, r) for p, r in zip(pinned, res)]
        for tk in tickets:
            assert fx.wait(tk, timeout_s=120)[0] == T.DONE
        st = fx.serve_stats()
    assert st["parts"] >= len(frames) and st["launches"] <= st["parts"]
    for r, rf in zip(res, ref):
        for k in rf:
            assert np.array_equal(r[k].numpy(), rf[k], equal_nan=k in ("state", "cov")), k
