"""CUDA fit with seed iteration (refits seeded from the fitted state) vs the
FP64 oracle, element by element through the C-ABI, with the fit's tolerances.

Seed iteration runs in the fit's variant instantiation (with energy loss);
the frames cover the default and a tight gate (clusters whose decision moves
between passes), a strong seed prior that iteration has to remove, and energy
loss and iteration together.
"""
import types

import numpy as np
import pytest

import oracle
import tpcgen
from parity import compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
PROTON = 0.938272


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_01205_gb300 as T
    from paper_2402_01205_gb300 import _build
    _build.build()
    return T


def fit_gpu(T, f, **cfg):
    g = types.SimpleNamespace(**{k: torch.from_numpy(np.ascontiguousarray(getattr(f, k))).cuda()
                                 for k in ("offsets", "x", "y", "z", "sy2", "sz2", "row")})
    with T.Fitter(**cfg) as fx:
        res = fx.fit(g)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in res.items()}


def check(f, gpu, orc, chi2_max=16.0, min_compared=0.97):
    rep = compare(f.offsets, gpu, orc, chi2_max=chi2_max)
    print(rep.summary())
    assert not rep.status_mismatch, rep.status_mismatch[:10]
    assert not rep.accept_mismatch, rep.accept_mismatch[:10]
    assert rep.ndf_mismatch == 0
    assert rep.max_state < 1e-3, rep.worst
    assert rep.max_cov < 1e-4, rep.worst
    assert rep.max_chi2 < 1e-4, rep.worst
    n_ok = int(((gpu["status"] == 0) & (orc["status"] == 0)).sum())
    assert rep.n_compared >= min_compared * n_ok
    return rep


@pytest.mark.parametrize("iterations,chi2_max", [(2, 16.0), (1, 9.0), (3, 9.0)])
def test_parity_with_seed_iteration(T, iterations, chi2_max):
    f = tpcgen.generate("detector50k", n_tracks=20_011, seed=51)
    gpu = fit_gpu(T, f, fit_iterations=iterations, chi2_max=chi2_max)
    orc = oracle.fit(f, oracle.FitConfig(xx0=5e-4, chi2_max=chi2_max, iterations=iterations), diagnostics=True)
    check(f, gpu, orc, chi2_max=chi2_max)
    plain = fit_gpu(T, f, chi2_max=chi2_max)
    assert not np.array_equal(plain["accept"], gpu["accept"])  # the passes were really repeated


@pytest.mark.parametrize("iterations", [0, 4])
def test_parity_with_a_strong_seed_prior(T, iterations):
    """Seed variances as small as one cluster's: without iteration the prior
    pulls the fit towards its three-point seed, with iteration it is removed;
    GPU and oracle agree either way."""
    strong = (0.01, 0.01, 1e-4, 1e-4, 1e-2)
    f = tpcgen.generate("detector50k", n_tracks=10_007, seed=52)
    gpu = fit_gpu(T, f, fit_iterations=iterations, seed_cov=strong)
    orc = oracle.fit(f, oracle.FitConfig(xx0=5e-4, seed_cov=strong, iterations=iterations), diagnostics=True)
    check(f, gpu, orc)


def test_parity_with_energy_loss_and_seed_iteration(T):
    f = tpcgen.generate("detector50k", n_tracks=10_009, seed=53, mass=PROTON, xrho=0.01, pt_min=0.3, pt_max=5.0)
    gpu = fit_gpu(T, f, xrho_per_row=0.01, mass_gev=PROTON, fit_iterations=1)
    orc = oracle.fit(f, oracle.FitConfig(xx0=5e-4, xrho=0.01, mass=PROTON, iterations=1), diagnostics=True)
    check(f, gpu, orc)
