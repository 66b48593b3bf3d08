"""GPU-vs-oracle comparison with the tolerances of the fit's precision split.

Tolerances of the parity bar:
  state      |dp_i| / max(sqrt(C_ii oracle), 1000 ulp32(p_i)) < 1e-3, where
             ulp32(p_i) is the spacing of binary32 numbers at the oracle's
             p_i: the library reports the state in binary32, which cannot
             come closer to p_i than half that spacing (this floor binds
             only when sigma_i < 1000 ulp32(p_i), e.g. sigma_z < 0.015 cm at
             |z| = 250 cm)
  covariance |dC_ij| / sqrt(C_ii C_jj)  < 1e-4   (normalised by the diagonal)
  chi2       |dchi2| <= 1e-4 * max(chi2, 1)
  ndf, status, accept bytes: identical, except that a track whose accept flag
  differs at a cluster whose oracle chi2 lies within 1e-5 (relative) of the
  gate is excluded from the comparison and counted.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TOL_STATE = 1e-3
TOL_COV = 1e-4
TOL_CHI2 = 1e-4
GATE_WINDOW = 1e-5


def _np(a):
    if hasattr(a, "detach"):
        return a.detach().cpu().numpy()
    return np.asarray(a)


@dataclass
class ParityReport:
    n_tracks: int = 0
    n_compared: int = 0
    n_gate_excluded: int = 0
    status_mismatch: list = field(default_factory=list)
    accept_mismatch: list = field(default_factory=list)
    max_state: float = 0.0
    max_cov: float = 0.0
    max_chi2: float = 0.0
    ndf_mismatch: int = 0
    worst: dict = field(default_factory=dict)

    @property
    def ok(self) -> bool:
        return (not self.status_mismatch and not self.accept_mismatch and self.ndf_mismatch == 0
                and self.max_state < TOL_STATE and self.max_cov < TOL_COV and self.max_chi2 < TOL_CHI2)

    def summary(self) -> str:
        return (f"tracks {self.n_tracks} compared {self.n_compared} gate-excluded {self.n_gate_excluded} "
                f"status-mismatch {len(self.status_mismatch)} accept-mismatch {len(self.accept_mismatch)} "
                f"ndf-mismatch {self.ndf_mismatch} max|dp|/sigma {self.max_state:.3e} "
                f"max cov {self.max_cov:.3e} max chi2 {self.max_chi2:.3e}")


def compare(offsets, gpu: dict, orc: dict, chi2_max: float = 16.0, track_ids=None) -> ParityReport:
    """``orc`` comes from oracle.fit(..., diagnostics=True) on the same frame.
    Without the diagnostics (no per-cluster chi2) every accept difference
    counts as a mismatch: the gate window cannot be checked."""
    off = _np(offsets).astype(np.int64)
    g = {k: _np(v) for k, v in gpu.items()}
    nt = off.shape[0] - 1
    rep = ParityReport(n_tracks=nt)
    ids = np.arange(nt) if track_ids is None else np.asarray(track_ids)
    gs, os_ = g["status"][ids], orc["status"][ids]
    bad = np.nonzero(gs != os_)[0]
    rep.status_mismatch = [(int(ids[i]), int(gs[i]), int(os_[i])) for i in bad]
    both_ok = ids[(gs == 0) & (os_ == 0)]
    keep = []
    for t in both_ok:
        a, b = off[t], off[t + 1]
        d = g["accept"][a:b] ^ orc["accept"][a:b]
        if not d.any():
            keep.append(t)
            continue
        # first differing decision in processing order: outward (ascending), then inward (descending)
        dout, din = (d & 1) != 0, (d & 2) != 0
        if "chi2_out_c" not in orc:
            rep.accept_mismatch.append(int(t))
            continue
        if dout.any():
            k, c = a + int(np.argmax(dout)), orc["chi2_out_c"]
        else:
            k, c = b - 1 - int(np.argmax(din[::-1])), orc["chi2_in_c"]
        if np.isfinite(c[k]) and abs(c[k] - chi2_max) <= GATE_WINDOW * chi2_max:
            rep.n_gate_excluded += 1
        else:
            rep.accept_mismatch.append(int(t))
    keep = np.asarray(keep, dtype=np.int64)
    rep.n_compared = int(keep.shape[0])
    if rep.n_compared == 0:
        return rep
    import oracle
    C = oracle.unpack_cov(orc["cov"][keep])
    sig = np.sqrt(np.diagonal(C, axis1=1, axis2=2))
    ulp32 = np.spacing(np.abs(orc["state"][keep]).astype(np.float32)).astype(np.float64)
    ds = np.abs(g["state"][keep].astype(np.float64) - orc["state"][keep]) / np.maximum(sig, 1000.0 * ulp32)
    Cg = oracle.unpack_cov(g["cov"][keep].astype(np.float64))
    dc = np.abs(Cg - C) / (sig[:, :, None] * sig[:, None, :])
    dchi = np.abs(g["chi2"][keep] - orc["chi2"][keep]) / np.maximum(orc["chi2"][keep], 1.0)
    rep.max_state = float(ds.max())
    rep.max_cov = float(dc.max())
    rep.max_chi2 = float(dchi.max())
    rep.ndf_mismatch = int((g["ndf"][keep] != orc["ndf"][keep]).sum())
    rep.worst = dict(state_track=int(keep[np.argmax(ds.max(1))]), cov_track=int(keep[np.argmax(dc.max((1, 2)))]),
                     chi2_track=int(keep[np.argmax(dchi)]))
    return rep


def compare_smoothed(offsets, status_ok, gpu_state, gpu_cov, orc_state, orc_cov) -> dict:
    """Per-cluster smoothed states of the tracks ``status_ok`` (bool per track)
    against the oracle's, with the bars of ``compare``: state over the
    oracle's sigma (with the binary32 floor), covariance over the square roots
    of the oracle's diagonal."""
    import oracle
    off = _np(offsets).astype(np.int64)
    ok = np.repeat(np.asarray(status_ok, bool), np.diff(off))
    gs, gc = _np(gpu_state).reshape(-1, 5)[ok].astype(np.float64), _np(gpu_cov).reshape(-1, 15)[ok].astype(np.float64)
    os_, oc = np.asarray(orc_state)[ok], np.asarray(orc_cov)[ok]
    C = oracle.unpack_cov(oc)
    sig = np.sqrt(np.diagonal(C, axis1=1, axis2=2))
    ulp32 = np.spacing(np.abs(os_).astype(np.float32)).astype(np.float64)
    ds = np.abs(gs - os_) / np.maximum(sig, 1000.0 * ulp32)
    dc = np.abs(oracle.unpack_cov(gc) - C) / (sig[:, :, None] * sig[:, None, :])
    return {"clusters": int(ok.sum()), "max_state": float(ds.max()) if ds.size else 0.0,
            "max_cov": float(dc.max()) if dc.size else 0.0,
            "q999_state": float(np.quantile(ds.max(1), 0.999)) if ds.size else 0.0,
            "q999_cov": float(np.quantile(dc.max((1, 2)), 0.999)) if dc.size else 0.0,
            "finite": bool(np.isfinite(gs).all() and np.isfinite(gc).all())}
