"""The two-filter smoother variant of the CUDA fit vs the FP64 oracle's
smoother (oracle_smooth), through the C-ABI: track outputs element by element
with the fit's bars, and the smoothed state and covariance at every cluster of
every fitted track.

The per-cluster bars are looser than the fit's: the combination weighs the
two filters' estimates by the inverse of C- + C+, whose correlation matrix
reaches condition numbers of 1e4 inside a track, and both filters keep their
covariances in binary32.  Combining the binary32 filters' outputs even in
FP64 leaves differences to the FP64 oracle of up to 2e-2 sigma (state) and
5.5e-3 (covariance over the square roots of its diagonal) at the worst of
millions of clusters, 1.8e-3 sigma at the 99.9th percentile (measured on the
GPU: 2.4e-2 and 4.2e-3 on 2.4 M clusters); the bars are 5e-2 and 1e-2.  For the compression residuals that consume the smoothed
states (codes of 0.01 cm against cluster errors of about 0.1 cm) that is far
below one code."""
import types

import numpy as np
import pytest

import oracle
import tpcgen
from parity import compare, compare_smoothed

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


def dev_frame(f):
    return types.SimpleNamespace(**{k: torch.from_numpy(np.ascontiguousarray(getattr(f, k))).cuda()
                                    for k in ("offsets", "x", "y", "z", "sy2", "sz2", "row")})


def smooth_gpu(T, f, **cfg):
    with T.Fitter(**cfg) as fx:
        res = T.alloc_result(f.n_tracks, f.n_clusters, device="cuda", smoothed=True)
        fx.fit(dev_frame(f), res)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in res.items()}


SM_STATE, SM_COV = 5e-2, 1e-2


def check(f, gpu, orc, min_ok=0.98):
    rep = compare(f.offsets, gpu, orc)
    print(rep.summary())
    assert not rep.status_mismatch, rep.status_mismatch[:10]
    assert not rep.accept_mismatch, rep.accept_mismatch[:10]
    assert rep.ndf_mismatch == 0
    assert rep.max_state < 1e-3 and rep.max_cov < 1e-4 and rep.max_chi2 < 1e-4, rep.worst
    ok = (gpu["status"] == 0) & (orc["status"] == 0)
    assert ok.mean() > min_ok
    sm = compare_smoothed(f.offsets, ok, gpu["smoothed_state"], gpu["smoothed_cov"], orc["sm_state"], orc["sm_cov"])
    print(sm)
    assert sm["finite"] and sm["max_state"] < SM_STATE and sm["max_cov"] < SM_COV, sm
    # clusters of tracks the fit did not complete carry NaN, as in the oracle
    stopped = np.repeat(~np.isin(orc["status"], (0, 7)), np.diff(f.offsets))
    assert np.array_equal(np.isnan(gpu["smoothed_state"][stopped]), np.isnan(orc["sm_state"][stopped]))


@pytest.mark.parametrize("preset,kw", [("sector1k", dict(n_tracks=1_000)), ("detector50k", dict(n_tracks=30_011)),
                                       ("pbpb2m", dict(n_tracks=100_003))])
def test_smoother_matches_oracle(T, preset, kw):
    f = tpcgen.generate(preset, seed=11, **kw)
    xx0 = 0.0 if preset == "sector1k" else 5e-4
    gpu = smooth_gpu(T, f, xx0_per_row=xx0)
    orc = oracle.smooth(f, oracle.FitConfig(xx0=xx0))
    check(f, gpu, orc)


def test_smoother_with_256_pad_rows(T):
    """Tracks of up to 255 clusters: the forward predictions fill every slot of
    the prediction scratch, which is sized by the handle's pad rows."""
    f = tpcgen.generate("detector50k", n_tracks=10_007, seed=14, n_rows=256, row_pitch=0.625)
    assert np.diff(f.offsets).max() >= 250
    gpu = smooth_gpu(T, f, n_rows=256, row_pitch_cm=0.625)
    check(f, gpu, oracle.smooth(f, oracle.FitConfig(n_rows=256, row_pitch=0.625)))


def test_smoother_with_unequal_variances_and_edge_cases(T):
    f = tpcgen.generate("detector50k", n_tracks=20_011, seed=12, var_mode=1)
    gpu = smooth_gpu(T, f)
    check(f, gpu, oracle.smooth(f, oracle.FitConfig()))
    g = tpcgen.generate("detector50k", n_tracks=40, seed=4)
    y, row = g.y.copy(), g.row.copy()
    y[g.offsets[1] + 5] = np.nan                   # NONFINITE
    row[g.offsets[2] + 7] = row[g.offsets[2] + 6]  # BAD_INPUT
    bad = tpcgen.Frame(g.offsets, g.x, y, g.z, g.sy2, g.sz2, row, g.sector)
    gb = smooth_gpu(T, bad)
    ob = oracle.smooth(bad, oracle.FitConfig())
    assert list(gb["status"][1:3]) == list(ob["status"][1:3]) == [4, 5]
    check(bad, gb, ob, min_ok=0.9)


def test_smoother_in_a_batch_graph_and_its_errors(T):
    f = tpcgen.generate("detector50k", n_tracks=10_000, seed=13)
    ref = smooth_gpu(T, f)
    d = dev_frame(f)
    with T.Fitter() as fx:
        res = T.alloc_result(f.n_tracks, f.n_clusters, device="cuda", smoothed=True)
        with T.Batch(fx, d, res) as b:
            b.launch()
            b.sync()
        got = {k: v.cpu().numpy() for k, v in res.items()}
        for k in ref:
            assert np.array_equal(ref[k], got[k], equal_nan=True), k
        host = T.alloc_result(f.n_tracks, f.n_clusters, smoothed=True)
        with pytest.raises(T.TpcfitError) as ei:
            fx.fit(f, host)  # a host frame cannot be smoothed
        assert ei.value.code == T.E_INVAL
    with T.Fitter(xrho_per_row=0.01) as fx:
        with pytest.raises(T.TpcfitError) as ei:
            fx.fit(d, T.alloc_result(f.n_tracks, f.n_clusters, device="cuda", smoothed=True))
        assert ei.value.code == T.E_INVAL
