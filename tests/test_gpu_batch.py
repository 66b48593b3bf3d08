"""Batched uneven events: one captured launch sequence over many events.

The batch graph must give exactly the results of a plain fit of the same
frame, agree with the FP64 oracle, see new contents of its buffers at every
replay, report malformed offsets at every replay, and give the same results
as one plain fit per event.
"""
import types

import numpy as np
import pytest

import oracle
import tpcgen
from parity import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KEYS = ("state", "cov", "x_ref", "chi2", "ndf", "status", "accept")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_01205_gb300 as T
    from paper_2402_01205_gb300 import _build
    _build.build()
    return T


@pytest.fixture(scope="module")
def events():
    return tpcgen.event_batch(n_events=96, median=120, sigma_ln=1.0, lo=10, hi=2000, seed=5)


def dev_frame(f):
    g = types.SimpleNamespace()
    for k in ("offsets", "x", "y", "z", "sy2", "sz2", "row"):
        setattr(g, k, torch.from_numpy(np.ascontiguousarray(getattr(f, k))).cuda())
    return g


def host(res):
    return {k: res[k].cpu().numpy() for k in KEYS}


def same(a, b):
    for k in KEYS:
        assert np.array_equal(a[k], b[k], equal_nan=k in ("state", "cov")), k


def test_batch_graph_equals_plain_fit_and_oracle(T, events):
    f, ev = events
    g = dev_frame(f)
    with T.Fitter() as fx:
        plain = host(fx.fit(g))
        with T.Batch(fx, g) as b:
            for _ in range(3):  # replays are independent
                b.launch()
            b.sync(timeout_s=60)
            same(plain, host(b.res))
    orc = oracle.fit(f, oracle.FitConfig(xx0=5e-4), diagnostics=True)
    rep = compare(f.offsets, plain, orc)
    print(rep.summary())
    assert not rep.status_mismatch and not rep.accept_mismatch and rep.ndf_mismatch == 0
    assert rep.max_state < 1e-3 and rep.max_cov < 1e-4 and rep.max_chi2 < 1e-4


def test_batch_equals_one_fit_per_event(T, events):
    f, ev = events
    g = dev_frame(f)
    with T.Fitter() as fx, T.Batch(fx, g) as b:
        b.launch()
        b.sync(timeout_s=60)
        whole = host(b.res)
        for e in (0, 1, 17, len(ev) - 2):
            t0, t1 = int(ev[e]), int(ev[e + 1])
            one = host(fx.fit(dev_frame(f.subset(t0, t1))))
            a, z = int(f.offsets[t0]), int(f.offsets[t1])
            for k in KEYS:
                w = whole[k][a:z] if k == "accept" else whole[k][t0:t1]
                assert np.array_equal(w, one[k], equal_nan=k in ("state", "cov")), (e, k)


def test_batch_replay_sees_new_contents_and_reports_bad_offsets(T, events):
    f, ev = events
    g = dev_frame(f)
    shifted = tpcgen.Frame(f.offsets, f.x, (f.y + np.float32(0.05)).astype(np.float32), f.z, f.sy2, f.sz2, f.row,
                           f.sector)
    with T.Fitter() as fx, T.Batch(fx, g) as b:
        ref_shift = host(fx.fit(dev_frame(shifted)))
        g.y.copy_(torch.from_numpy(shifted.y))
        b.launch()
        b.sync(timeout_s=60)
        same(ref_shift, host(b.res))
        # malformed offsets: reported by the replay that sees them, then cleared
        o50 = g.offsets[50].clone()
        g.offsets[50] = g.offsets[52]
        b.launch()
        with pytest.raises(T.TpcfitError) as ei:
            b.sync(timeout_s=60)
        assert ei.value.code == T.E_INVAL
        g.offsets[50] = o50
        b.launch()
        b.sync(timeout_s=60)
        same(ref_shift, host(b.res))


def test_batch_on_caller_stream_and_block_shapes(T, events):
    f, ev = events
    g = dev_frame(f)
    with T.Fitter() as fx:
        ref = host(fx.fit(g))
    s = torch.cuda.Stream()
    for bt, bps in ((128, 0), (128, 4), (128, 3), (256, 1), (256, 0)):
        with T.Fitter(block_threads=bt, blocks_per_sm=bps) as fx, T.Batch(fx, g) as b:
            b.launch(stream=s)
            b.sync(timeout_s=60)
            same(ref, host(b.res))


def test_batch_rejects_host_frames(T, events):
    f, ev = events
    with T.Fitter() as fx:
        with pytest.raises(T.TpcfitError) as ei:
            T.Batch(fx, f.subset(0, 10), T.alloc_result(10, int(f.offsets[10])))
        assert ei.value.code == T.E_INVAL


def test_batch_graph_of_the_fit_variant_equals_its_plain_fit(T, events):
    """The graph-captured sequence launches the variant instantiation when the
    handle's configuration asks for it (energy loss, seed iteration)."""
    f, ev = events
    g = dev_frame(f)
    with T.Fitter(xrho_per_row=0.01, fit_iterations=1) as fx:
        plain = host(fx.fit(g))
        with T.Batch(fx, g) as b:
            b.launch()
            b.sync(timeout_s=60)
            same(plain, host(b.res))
    with T.Fitter(xrho_per_row=0.01, fit_iterations=1, blocks_per_sm=5) as fx:  # the variant's grid is cut to 4
        same(plain, host(fx.fit(g)))
    with T.Fitter() as fx:
        assert not np.array_equal(host(fx.fit(g))["state"], plain["state"])
