"""FP64 CPU oracle for the batched TPC Kalman track fit.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library never does.
It shares no code, header, table or constant with the CUDA library.

``kalman_oracle.c`` is the plain FP64 Kalman fitter (seed, exact-helix
propagation, chi2-gated update, Highland scattering, outward then inward pass).
``lsq.py`` is an independent linearised global least-squares fitter used to
pin it.  The paper (Sec. 5, Sec. 6) names full TPC tracking as the GPU hot
path but does not write the fit out; the formulas follow the textbook Kalman
filter for track fitting (Fruhwirth 1987) and the PDG Highland formula.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kalman_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

KB = 0.299792458e-2
STATUS = {0: "OK", 1: "TOO_FEW", 2: "SNP_LIMIT", 3: "NOT_PD", 4: "NONFINITE", 5: "BAD_INPUT", 6: "STOPPED",
          7: "DERAILED"}


def build(force: bool = False) -> str:
    """Compile the oracle into an in-tree shared library (plain gcc -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(ctypes.Structure):
    _fields_ = [("bz", ctypes.c_double), ("chi2_max", ctypes.c_double), ("xx0", ctypes.c_double),
                ("mass", ctypes.c_double), ("snp_max", ctypes.c_double), ("seed_cov", ctypes.c_double * 5),
                ("min_clusters", ctypes.c_int32), ("n_rows", ctypes.c_int32), ("row_x", ctypes.c_void_p),
                ("restart_scale", ctypes.c_double), ("xrho", ctypes.c_double), ("eloss_za", ctypes.c_double),
                ("eloss_i", ctypes.c_double), ("n_iterations", ctypes.c_int32), ("reseed_pct", ctypes.c_int32),
                ("derail_pct", ctypes.c_int32)]


class _Res(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("state", "cov", "x_ref", "chi2", "ndf", "status", "accept", "chi2_out_c", "chi2_in_c", "state_in_c",
                 "state_out_t", "restart_t")]


class _FollowCfg(ctypes.Structure):
    _fields_ = [("window_sigma", ctypes.c_double), ("nominal_v", ctypes.c_double), ("max_miss", ctypes.c_int32),
                ("tan_edge", ctypes.c_double), ("z_max", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_fit.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 7 + \
            [ctypes.POINTER(_Res), ctypes.c_int]
        lib.oracle_fit.restype = ctypes.c_int
        lib.orc_propagate.argtypes = [_D, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D]
        lib.orc_propagate.restype = ctypes.c_int
        lib.orc_update.argtypes = [_D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, _D, ctypes.POINTER(ctypes.c_int)]
        lib.orc_update.restype = ctypes.c_int
        lib.orc_ms_noise.argtypes = [_D, _D, ctypes.c_double, ctypes.c_double]
        lib.orc_seed.argtypes = [_D, _D, _D, ctypes.c_double, _D]
        lib.orc_dedx.argtypes = [ctypes.c_double] * 4
        lib.orc_dedx.restype = ctypes.c_double
        lib.orc_eloss.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Cfg), ctypes.c_double]
        lib.orc_eloss.restype = ctypes.c_int
        lib.oracle_residuals.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int64] * 2 + [ctypes.c_void_p] * 11
        lib.oracle_follow.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(_FollowCfg), ctypes.c_int64] + \
            [ctypes.c_void_p] * 6 + [ctypes.c_int64] + [ctypes.c_void_p] * 10 + [ctypes.c_int]
        lib.oracle_follow.restype = ctypes.c_int
        lib.oracle_residuals.restype = ctypes.c_int
        lib.oracle_smooth.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 7 + \
            [ctypes.POINTER(_Res), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.oracle_smooth.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class FitConfig:
    """Fit parameters (readings of the method; the paper gives none)."""
    bz: float = 0.5
    chi2_max: float = 16.0
    xx0: float = 5e-4
    mass: float = 0.13957
    snp_max: float = 0.999
    seed_cov: tuple = (1.0, 1.0, 0.01, 0.01, 1.0)
    min_clusters: int = 10
    restart_scale: float = 100.0
    n_rows: int = 152
    row_x0: float = 85.0
    row_pitch: float = 162.0 / 151.0
    xrho: float = 0.0          # energy-loss layer per crossed row, g/cm^2 (0: none)
    eloss_za: float = 0.49555  # its Z/A (neon)
    eloss_i_ev: float = 137.0  # its mean excitation energy, eV (neon)
    iterations: int = 0        # refits seeded from the previous fit's state
    reseed_pct: int = 50       # inward re-seed below this outward acceptance (percent of the clusters)
    derail_pct: int = 80       # a fit whose inward pass accepted fewer (percent) is DERAILED

    def row_x(self) -> np.ndarray:
        return (self.row_x0 + np.arange(self.n_rows, dtype=np.float64) * self.row_pitch).astype(np.float32)


def _cfg_struct(cfg: "FitConfig", rx: np.ndarray) -> _Cfg:
    return _Cfg(cfg.bz, cfg.chi2_max, cfg.xx0, cfg.mass, cfg.snp_max, (ctypes.c_double * 5)(*cfg.seed_cov),
                cfg.min_clusters, cfg.n_rows, rx.ctypes.data, cfg.restart_scale, cfg.xrho, cfg.eloss_za,
                cfg.eloss_i_ev * 1e-9, cfg.iterations, cfg.reseed_pct, cfg.derail_pct)


def dedx(p: float, mass: float, za: float = 0.49555, i_ev: float = 137.0) -> float:
    """Mean stopping power (Bethe formula, no density effect) in GeV cm^2/g (orc_dedx)."""
    lib = _load()
    return float(lib.orc_dedx(float(p), float(mass), float(za), float(i_ev) * 1e-9))


def eloss_step(state, cov, cfg: "FitConfig", direction: float):
    """One energy-loss layer applied to (state, 5x5 cov) as the fit applies it
    (orc_eloss); returns (status, state, cov)."""
    lib = _load()
    p = np.ascontiguousarray(state, dtype=np.float64).copy()
    C = np.ascontiguousarray(cov, dtype=np.float64).copy()
    rx = cfg.row_x()
    c = _cfg_struct(cfg, rx)
    st = lib.orc_eloss(p.ctypes.data, C.ctypes.data, ctypes.byref(c), ctypes.c_double(direction))
    return int(st), p, C


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def fit(frame, cfg: Optional[FitConfig] = None, threads: Optional[int] = None, diagnostics: bool = False) -> dict:
    """Fit every track of ``frame`` (any object with offsets/x/y/z/sy2/sz2/row arrays)."""
    lib = _load()
    cfg = cfg or FitConfig()
    off = np.ascontiguousarray(frame.offsets, dtype=np.int64)
    arrs = [np.ascontiguousarray(getattr(frame, k), dtype=np.float32) for k in ("x", "y", "z", "sy2", "sz2")]
    row = np.ascontiguousarray(frame.row, dtype=np.uint8)
    nt, nc = off.shape[0] - 1, int(arrs[0].shape[0])
    rx = cfg.row_x()
    c = _cfg_struct(cfg, rx)
    out = dict(state=np.zeros((nt, 5)), cov=np.zeros((nt, 15)), x_ref=np.zeros(nt), chi2=np.zeros(nt),
               ndf=np.zeros(nt, np.int32), status=np.zeros(nt, np.int32), accept=np.zeros(nc, np.uint8))
    if diagnostics:
        out.update(chi2_out_c=np.zeros(nc), chi2_in_c=np.zeros(nc), state_in_c=np.zeros((nc, 5)),
                   state_out_t=np.full((nt, 5), np.nan), restart_t=np.full((nt, 5), np.nan))
    r = _Res(*[out[k].ctypes.data if k in out else None for k, _ in _Res._fields_])
    th = threads if threads else (os.cpu_count() or 1)
    rc = lib.oracle_fit(ctypes.byref(c), nt, nc, off.ctypes.data, *[a.ctypes.data for a in arrs], row.ctypes.data,
                        ctypes.byref(r), th)
    if rc != 0:
        raise ValueError("oracle_fit: malformed track offsets")
    out["threads"] = min(th, max(nt, 1))
    return out


def smooth(frame, cfg: Optional[FitConfig] = None, threads: Optional[int] = None) -> dict:
    """Two-filter smoother (oracle_smooth): the track outputs of the smoothed
    fit (state and covariance at the innermost cluster, chi2, ndf, status,
    accept flags), the smoothed state ``sm_state`` (nc, 5) and packed
    covariance ``sm_cov`` (nc, 15) at every cluster, and the backward
    filter's starting state ``state_out_t`` and covariance diagonal
    ``restart_t`` per track."""
    lib = _load()
    cfg = cfg or FitConfig()
    if cfg.xrho > 0 or cfg.iterations > 0:
        raise ValueError("the smoother takes neither energy loss nor seed iteration")
    off = np.ascontiguousarray(frame.offsets, dtype=np.int64)
    arrs = [np.ascontiguousarray(getattr(frame, k), dtype=np.float32) for k in ("x", "y", "z", "sy2", "sz2")]
    row = np.ascontiguousarray(frame.row, dtype=np.uint8)
    nt, nc = off.shape[0] - 1, int(arrs[0].shape[0])
    rx = cfg.row_x()
    c = _cfg_struct(cfg, rx)
    out = dict(state=np.zeros((nt, 5)), cov=np.zeros((nt, 15)), x_ref=np.zeros(nt), chi2=np.zeros(nt),
               ndf=np.zeros(nt, np.int32), status=np.zeros(nt, np.int32), accept=np.zeros(nc, np.uint8),
               sm_state=np.zeros((nc, 5)), sm_cov=np.zeros((nc, 15)),
               state_out_t=np.full((nt, 5), np.nan), restart_t=np.full((nt, 5), np.nan))
    r = _Res(*[out[k].ctypes.data if k in out else None for k, _ in _Res._fields_])
    th = threads if threads else (os.cpu_count() or 1)
    rc = lib.oracle_smooth(ctypes.byref(c), nt, nc, off.ctypes.data, *[a.ctypes.data for a in arrs],
                           row.ctypes.data, ctypes.byref(r), out["sm_state"].ctypes.data, out["sm_cov"].ctypes.data, th)
    if rc != 0:
        raise ValueError("oracle_smooth: malformed track offsets")
    return out


def residuals(frame, fitted: dict, step=(0.01, 0.01), bz: float = 0.5) -> dict:
    """Track-model compression residual codes of ``frame`` against the oracle's
    own fit ``fitted`` (the output of ``fit``): int16 codes ``res_y``,
    ``res_z`` and the unquantised residuals in code units ``raw_y``, ``raw_z``."""
    lib = _load()
    off = np.ascontiguousarray(frame.offsets, dtype=np.int64)
    x, y, z = (np.ascontiguousarray(getattr(frame, k), dtype=np.float32) for k in ("x", "y", "z"))
    nt, nc = off.shape[0] - 1, int(x.shape[0])
    st = np.ascontiguousarray(fitted["state"], dtype=np.float64)
    xr = np.ascontiguousarray(fitted["x_ref"], dtype=np.float64)
    status = np.ascontiguousarray(fitted["status"], dtype=np.int32)
    out = dict(res_y=np.zeros(nc, np.int16), res_z=np.zeros(nc, np.int16), raw_y=np.zeros(nc), raw_z=np.zeros(nc))
    rc = lib.oracle_residuals(bz, step[0], step[1], nt, nc, off.ctypes.data, x.ctypes.data, y.ctypes.data,
                              z.ctypes.data, st.ctypes.data, xr.ctypes.data, status.ctypes.data,
                              *[out[k].ctypes.data for k in ("res_y", "res_z", "raw_y", "raw_z")])
    if rc != 0:
        raise ValueError("oracle_residuals: malformed track offsets")
    return out


@dataclass
class FollowConfig:
    """Track-following readings (the paper describes no algorithm)."""
    window_sigma: float = 4.0      # search window half-width in sigma
    nominal_v: float = 0.01        # cluster variance used for the window (cm^2)
    max_miss: int = 4              # consecutive rows without a cluster that end the track
    tan_edge: float = float(np.tan(np.radians(10.0)))  # sector edge
    z_max: float = 250.0
    seed_cov: tuple = (0.01, 0.01, 1e-4, 1e-4, 0.01)


def cluster_sectors(frame) -> np.ndarray:
    """Sector of every cluster (the frames store one sector per track)."""
    return np.repeat(np.asarray(frame.sector, dtype=np.uint8), np.diff(frame.offsets)).astype(np.uint8)


def follow(hits, seeds: dict, cfg: Optional[FitConfig] = None, fcfg: Optional[FollowConfig] = None,
           threads: Optional[int] = None) -> dict:
    """Follow ``seeds`` (dict: state float64[ns,5], row uint8[ns], sector uint8[ns]) through the
    clusters of ``hits`` (y, z, sy2, sz2, row arrays and ``sectors`` per cluster)."""
    lib = _load()
    cfg = cfg or FitConfig()
    fcfg = fcfg or FollowConfig()
    y, z, sy2, sz2 = (np.ascontiguousarray(getattr(hits, k), dtype=np.float32) for k in ("y", "z", "sy2", "sz2"))
    row = np.ascontiguousarray(hits.row, dtype=np.uint8)
    sec = np.ascontiguousarray(hits.sectors, dtype=np.uint8)
    st = np.ascontiguousarray(seeds["state"], dtype=np.float64)
    srow = np.ascontiguousarray(seeds["row"], dtype=np.uint8)
    ssec = np.ascontiguousarray(seeds["sector"], dtype=np.uint8)
    scov = np.ascontiguousarray(fcfg.seed_cov, dtype=np.float64)
    ns, nc, nr = st.shape[0], y.shape[0], cfg.n_rows
    rx = cfg.row_x()
    c = _cfg_struct(cfg, rx)
    fc = _FollowCfg(fcfg.window_sigma, fcfg.nominal_v, fcfg.max_miss, fcfg.tan_edge, fcfg.z_max)
    out = dict(att=np.zeros((ns, nr), np.int32), n_att=np.zeros(ns, np.int32), status=np.zeros(ns, np.int32),
               state=np.zeros((ns, 5)), best2=np.zeros((ns, nr, 2)), edge=np.zeros((ns, nr)))
    th = threads if threads else (os.cpu_count() or 1)
    rc = lib.oracle_follow(ctypes.byref(c), ctypes.byref(fc), nc, y.ctypes.data, z.ctypes.data, sy2.ctypes.data,
                           sz2.ctypes.data, row.ctypes.data, sec.ctypes.data, ns, st.ctypes.data, srow.ctypes.data,
                           ssec.ctypes.data, scov.ctypes.data, *[out[k].ctypes.data for k in
                                                                ("att", "n_att", "status", "state", "best2", "edge")],
                           th)
    if rc != 0:
        raise ValueError("oracle_follow: bad arguments")
    return out


def propagate(p1, x1: float, x2: float, bz: float = 0.5, snp_max: float = 0.999):
    """Exact-helix transport of a state between two pad-row planes; returns (status, p2, F)."""
    lib = _load()
    p1 = np.ascontiguousarray(p1, dtype=np.float64)
    p2 = np.zeros(5)
    F = np.zeros(25)
    st = lib.orc_propagate(_p(p1), x1, x2, bz, snp_max, _p(p2), _p(F))
    return st, p2, F.reshape(5, 5)


def update(p, C, yc, zc, sy2, sz2, chi2_max=16.0):
    """One gated Kalman update; returns (status, p, C, chi2, accepted)."""
    lib = _load()
    p = np.array(p, dtype=np.float64)
    C = np.array(C, dtype=np.float64).reshape(25).copy()
    chi2 = ctypes.c_double()
    acc = ctypes.c_int()
    st = lib.orc_update(_p(p), _p(C), yc, zc, sy2, sz2, chi2_max, ctypes.byref(chi2), ctypes.byref(acc))
    return st, p, C.reshape(5, 5), chi2.value, bool(acc.value)


def ms_noise(p, C, xx0: float, mass: float = 0.13957):
    """Covariance after adding one row's multiple-scattering noise."""
    lib = _load()
    p = np.array(p, dtype=np.float64)
    C = np.array(C, dtype=np.float64).reshape(25).copy()
    lib.orc_ms_noise(_p(p), _p(C), xx0, mass)
    return C.reshape(5, 5)


def seed(a, b, c, bz: float = 0.5):
    """Three-point seed state at point a (each point = (x, y, z))."""
    lib = _load()
    pa, pb, pc = (np.array(v, dtype=np.float64) for v in (a, b, c))
    p = np.zeros(5)
    lib.orc_seed(_p(pa), _p(pb), _p(pc), bz, _p(p))
    return p


def unpack_cov(c15: np.ndarray) -> np.ndarray:
    """Packed lower triangle (00,10,11,20,...) -> full symmetric (..., 5, 5)."""
    c15 = np.asarray(c15)
    out = np.zeros(c15.shape[:-1] + (5, 5), dtype=c15.dtype)
    k = 0
    for i in range(5):
        for j in range(i + 1):
            out[..., i, j] = c15[..., k]
            out[..., j, i] = c15[..., k]
            k += 1
    return out
