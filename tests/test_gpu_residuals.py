"""Track-model compression residual codes: CUDA path against the FP64 oracle.

The codes are integers decided from floating point: each side quantises its
own residual (GPU in FP32 from its fitted state, oracle in FP64 from its own).
The fitted states agree within the parity tolerance, which moves a residual by
far less than 0.05 code units here; so codes must be identical except where
the oracle's unquantised residual lies within 0.05 of a rounding boundary
(half-integer), and there they may differ by one.  Non-OK tracks carry the
not-encoded code -32768 on both sides.
"""
import types

import numpy as np
import pytest

import oracle
import tpcgen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WINDOW = 0.05


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_01205_gb300 as T
    from paper_2402_01205_gb300 import _build
    _build.build()
    return T


def dev_frame(f):
    g = types.SimpleNamespace()
    for k in ("offsets", "x", "y", "z", "sy2", "sz2", "row"):
        setattr(g, k, torch.from_numpy(np.ascontiguousarray(getattr(f, k))).cuda())
    return g


def gpu_fit(T, f, **cfg):
    with T.Fitter(**cfg) as fx:
        res = T.alloc_result(f.n_tracks, f.n_clusters, device="cuda", residuals=True)
        fx.fit(dev_frame(f), res)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in res.items()}


def check_codes(f, g, orc, q):
    per_cl = np.diff(f.offsets)
    both = np.repeat((g["status"] == 0) & (orc["status"] == 0), per_cl)
    for axis in ("y", "z"):
        cg, co, raw = g["res_" + axis], q["res_" + axis], q["raw_" + axis]
        frac = np.abs(np.abs(raw - np.floor(raw)) - 0.5)
        edge = both & (frac < WINDOW)
        diff = both & (cg != co)
        assert not np.any(diff & ~edge), np.nonzero(diff & ~edge)[0][:10]
        assert np.all(np.abs(cg[diff].astype(np.int32) - co[diff]) <= 1)
        print(f"{axis}: {both.sum()} clusters, {diff.sum()} differ at a rounding boundary "
              f"({edge.sum()} within {WINDOW} of one)")
    not_ok = np.repeat(g["status"] != 0, per_cl)
    assert np.all(g["res_y"][not_ok] == -32768) and np.all(g["res_z"][not_ok] == -32768)
    assert both.sum() > 0.95 * f.n_clusters


def test_residual_codes_match_oracle_detector(T):
    f = tpcgen.generate("detector50k", n_tracks=30_011, seed=8)
    g = gpu_fit(T, f)
    orc = oracle.fit(f, oracle.FitConfig(xx0=5e-4))
    check_codes(f, g, orc, oracle.residuals(f, orc))


def test_residual_codes_match_oracle_pbpb_spectrum_other_steps(T):
    f = tpcgen.generate("pbpb2m", n_tracks=40_000, seed=9)
    g = gpu_fit(T, f, res_step_y_cm=0.005, res_step_z_cm=0.02)
    orc = oracle.fit(f, oracle.FitConfig(xx0=5e-4))
    check_codes(f, g, orc, oracle.residuals(f, orc, step=(0.005, 0.02)))


def test_residuals_leave_the_fit_unchanged_and_agree_across_paths(T):
    f = tpcgen.generate("detector50k", n_tracks=12_000, seed=10)
    with_res = gpu_fit(T, f)
    with T.Fitter() as fx:
        plain = {k: v.cpu().numpy() for k, v in fx.fit(dev_frame(f)).items()}
    for k in plain:
        assert np.array_equal(plain[k], with_res[k], equal_nan=k in ("state", "cov")), k
    # host frame, chunked path
    with T.Fitter(host_chunk_clusters=200_000) as fx:
        host = fx.fit(f, T.alloc_result(f.n_tracks, f.n_clusters, residuals=True))
    # served frame, split into parts
    with T.Fitter(host_chunk_clusters=300_000, max_slots=2) as fx:
        pf = types.SimpleNamespace(**{k: torch.from_numpy(np.ascontiguousarray(getattr(f, k))).pin_memory()
                                      for k in ("offsets", "x", "y", "z", "sy2", "sz2", "row")})
        sr = T.alloc_result(f.n_tracks, f.n_clusters, pinned=True, residuals=True)
        assert fx.wait(fx.submit(pf, sr), 60)[0] == T.DONE
    for k in ("res_y", "res_z"):
        assert np.array_equal(with_res[k], host[k]), k
        assert np.array_equal(with_res[k], sr[k].numpy()), k
    # a batch graph writes them too
    g = dev_frame(f)
    res = T.alloc_result(f.n_tracks, f.n_clusters, device="cuda", residuals=True)
    with T.Fitter() as fx, T.Batch(fx, g, res) as b:
        b.launch()
        b.sync(60)
        for k in ("res_y", "res_z"):
            assert np.array_equal(with_res[k], res[k].cpu().numpy()), k


def test_noise_free_residuals_are_zero(T):
    f = tpcgen.generate("sector1k", n_tracks=500, sigma_y=0.0, sigma_z=0.0, seed=2)
    g = gpu_fit(T, f, xx0_per_row=0.0)
    assert np.all(g["status"] == 0)
    print("max |code|", np.abs(g["res_y"]).max(), np.abs(g["res_z"]).max())
    assert np.all(np.abs(g["res_y"]) <= 1) and np.all(np.abs(g["res_z"]) <= 1)
