"""The allocation-free entry point tpcfit_fit_noalloc, through the C-ABI.

Some callers cannot allocate device memory while they run: their GPU memory
is already owned by another allocator, or their steady-state processing loop
forbids allocation to keep latency predictable.  tpcfit_fit_noalloc serves
them from one static device scratch array of fixed size.  Its results must
equal those of tpcfit_fit on the same frames, also when calls follow one
another and reuse the shared array.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.
"""
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


def dev_frame(f):
    return types.SimpleNamespace(**{k: torch.from_numpy(np.ascontiguousarray(getattr(f, k))).cuda()
                                    for k in ("offsets", "x", "y", "z", "sy2", "sz2", "row")})


def host(res):
    return {k: v.cpu().numpy() for k, v in res.items()}


def assert_same_fit(got, ref):
    """Same tolerances as the oracle parity tests, with tpcfit_fit as reference."""
    assert np.array_equal(got["status"], ref["status"])
    assert np.array_equal(got["ndf"], ref["ndf"])
    assert np.array_equal(got["accept"], ref["accept"])
    assert np.array_equal(got["x_ref"], ref["x_ref"])
    ok = ref["status"] == 0
    import oracle
    C = oracle.unpack_cov(ref["cov"][ok].astype(np.float64))
    sig = np.sqrt(np.diagonal(C, axis1=1, axis2=2))
    ds = np.abs(got["state"][ok].astype(np.float64) - ref["state"][ok]) / sig
    Cg = oracle.unpack_cov(got["cov"][ok].astype(np.float64))
    dc = np.abs(Cg - C) / (sig[:, :, None] * sig[:, None, :])
    dchi = np.abs(got["chi2"][ok] - ref["chi2"][ok]) / np.maximum(ref["chi2"][ok], 1.0)
    assert ds.max() < 1e-3 and dc.max() < 1e-4 and dchi.max() < 1e-4


def test_noalloc_matches_fit_on_two_calls_in_a_row(T):
    fa = tpcgen.generate("detector50k", n_tracks=20_011, seed=31)
    fb = tpcgen.generate("pbpb2m", n_tracks=60_000, seed=32)
    da, db = dev_frame(fa), dev_frame(fb)
    with T.Fitter() as fx:
        ref_a, ref_b = host(fx.fit(da)), host(fx.fit(db))
    out_a = T.alloc_result(fa.n_tracks, fa.n_clusters, device="cuda")
    out_b = T.alloc_result(fb.n_tracks, fb.n_clusters, device="cuda")
    T.fit_noalloc(da, out_a)          # first call (also looks up the scratch address)
    T.fit_noalloc(db, out_b)          # second call reuses the shared scratch
    got_a, got_b = host(out_a), host(out_b)
    assert_same_fit(got_a, ref_a)
    assert_same_fit(got_b, ref_b)
    # the same frame again after a different one: nothing left over from the previous call
    out_a2 = T.alloc_result(fa.n_tracks, fa.n_clusters, device="cuda")
    T.fit_noalloc(da, out_a2)
    assert_same_fit(host(out_a2), ref_a)


def test_noalloc_rejects_frames_above_the_limit(T):
    f = tpcgen.generate("sector1k", n_tracks=65_537, seed=33)
    with pytest.raises(T.TpcfitError) as ei:
        T.fit_noalloc(dev_frame(f), T.alloc_result(f.n_tracks, f.n_clusters, device="cuda"))
    assert ei.value.code == T.E_INVAL
    assert "TPCFIT_NOALLOC_MAX_TRACKS" in str(ei.value)  # the detail of tpcfit_last_error_message
    assert torch.cuda.current_device() == 0  # the caller's device is current again


def test_noalloc_writes_the_residual_codes_of_fit(T):
    """Residual codes requested from the allocation-free call are those of
    tpcfit_fit on the same frame (same kernels, same inputs: bit for bit)."""
    f = tpcgen.generate("detector50k", n_tracks=9_001, seed=36)
    d = dev_frame(f)
    with T.Fitter() as fx:
        ref = T.alloc_result(f.n_tracks, f.n_clusters, device="cuda", residuals=True)
        fx.fit(d, ref)
        ref = host(ref)
    for _ in range(2):
        out = T.alloc_result(f.n_tracks, f.n_clusters, device="cuda", residuals=True)
        T.fit_noalloc(d, out)
        got = host(out)
        assert_same_fit(got, ref)
        assert np.array_equal(got["res_y"], ref["res_y"]) and np.array_equal(got["res_z"], ref["res_z"])


def test_noalloc_with_energy_loss_equals_fit(T):
    f = tpcgen.generate("detector50k", n_tracks=8_000, seed=34, mass=0.938272, xrho=0.01, pt_min=0.3, pt_max=5.0)
    d = dev_frame(f)
    with T.Fitter(xrho_per_row=0.01, mass_gev=0.938272) as fx:
        ref = host(fx.fit(d))
    out = T.alloc_result(f.n_tracks, f.n_clusters, device="cuda")
    T.fit_noalloc(d, out, T.default_config(xrho_per_row=0.01, mass_gev=0.938272))
    got = host(out)
    assert_same_fit(got, ref)
    assert np.array_equal(got["state"], ref["state"])  # same kernel, same inputs: bit-identical


def test_noalloc_with_seed_iteration_equals_fit(T):
    f = tpcgen.generate("detector50k", n_tracks=8_000, seed=35)
    d = dev_frame(f)
    with T.Fitter(fit_iterations=2) as fx:
        ref = host(fx.fit(d))
    out = T.alloc_result(f.n_tracks, f.n_clusters, device="cuda")
    T.fit_noalloc(d, out, T.default_config(fit_iterations=2))
    got = host(out)
    assert_same_fit(got, ref)
    assert np.array_equal(got["state"], ref["state"])
