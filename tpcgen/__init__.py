"""Seeded synthetic TPC time frames (inputs for tests and benchmarks only).

The generator itself is C (``helixgen.c``): helices in a uniform Bz field,
intersected with the pad-row planes of one sector frame as global circles,
with Gaussian cluster noise, Highland multiple-scattering kicks, dropout and
outliers.  These frames stand in for the ALICE Monte-Carlo / Pb-Pb time frames
that the paper measures on (Sec. 7); they are not available here.

This module holds no fitting arithmetic and is imported by both the oracle
tests and the CUDA-path tests/benchmarks as their common input source.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "helixgen.c")
_LIB_PATH = os.path.join(_HERE, "libhelixgen.so")
_lib = None

# TPC geometry shared by every workload: 152 pad rows from 85 to 247 cm.
N_ROWS = 152
ROW_X0 = 85.0
ROW_PITCH = 162.0 / 151.0


def build(force: bool = False) -> str:
    """Compile helixgen.c into an in-tree shared library (gcc, portable flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Config(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64), ("n_tracks", ctypes.c_int64),
        ("n_rows", ctypes.c_int32), ("min_clusters", ctypes.c_int32),
        ("row_x0", ctypes.c_double), ("row_pitch", ctypes.c_double),
        ("bz", ctypes.c_double), ("xx0", ctypes.c_double), ("mass", ctypes.c_double),
        ("sigma_y", ctypes.c_double), ("sigma_z", ctypes.c_double),
        ("p_drop", ctypes.c_double), ("p_outlier", ctypes.c_double), ("outlier_half", ctypes.c_double),
        ("pt_mode", ctypes.c_int32), ("n_phi_sectors", ctypes.c_int32),
        ("pt_min", ctypes.c_double), ("pt_max", ctypes.c_double), ("pt_mean", ctypes.c_double),
        ("sector_half_angle", ctypes.c_double), ("vtx_sigma", ctypes.c_double),
        ("tgl_max", ctypes.c_double), ("z_max", ctypes.c_double), ("snp_max", ctypes.c_double),
        ("max_attempts", ctypes.c_int32), ("n_threads", ctypes.c_int32),
        ("track_id_offset", ctypes.c_int64),
        ("xrho", ctypes.c_double), ("eloss_za", ctypes.c_double), ("eloss_i_ev", ctypes.c_double),
        ("var_mode", ctypes.c_int32), ("var_lo", ctypes.c_double), ("var_hi", ctypes.c_double),
    ]


class _Out(ctypes.Structure):
    _fields_ = [
        ("offsets", ctypes.c_void_p), ("counts", ctypes.c_void_p),
        ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
        ("sy2", ctypes.c_void_p), ("sz2", ctypes.c_void_p),
        ("row", ctypes.c_void_p), ("sector", ctypes.c_void_p),
        ("truth", ctypes.c_void_p), ("flags", ctypes.c_void_p), ("truth_vertex", ctypes.c_void_p),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.tpcgen_count.argtypes = [ctypes.POINTER(_Config), ctypes.c_void_p]
        lib.tpcgen_fill.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Out)]
        lib.tpcgen_lognormal_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        lib.tpcgen_poisson_arrivals.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p]
        _lib = lib
    return _lib


# Workload presets (sizes and distributions of the five synthetic workloads).
BASE = dict(
    n_rows=N_ROWS, row_x0=ROW_X0, row_pitch=ROW_PITCH, bz=0.5, mass=0.13957,
    sigma_y=0.1, sigma_z=0.1, pt_mode=0, pt_min=0.2, pt_max=10.0, pt_mean=0.6,
    sector_half_angle=math.radians(10.0), vtx_sigma=0.01, tgl_max=0.9, z_max=250.0,
    snp_max=0.99, min_clusters=10, max_attempts=1000,
    xrho=0.0, eloss_za=0.49555, eloss_i_ev=137.0,  # no energy loss unless xrho > 0 (neon material)
    var_mode=0, var_lo=0.002, var_hi=0.05,  # var_mode 1: per-cluster sy2, sz2 log-uniform in [var_lo, var_hi]
)
PRESETS = {
    # single sector, 1,000 tracks, no scattering / dropout / outliers
    "sector1k": dict(BASE, n_tracks=1000, xx0=0.0, p_drop=0.0, p_outlier=0.0, outlier_half=2.0, n_phi_sectors=1),
    # full 36-sector detector, 50,000 tracks, scattering + 5% dropout + 1% outliers
    "detector50k": dict(BASE, n_tracks=50_000, xx0=5e-4, p_drop=0.05, p_outlier=0.01, outlier_half=2.0,
                        n_phi_sectors=18),
    # Pb-Pb-scale frame: 2,000,000 tracks, exponential pT spectrum (mean 0.6, floor 0.05)
    "pbpb2m": dict(BASE, n_tracks=2_000_000, xx0=5e-4, p_drop=0.05, p_outlier=0.01, outlier_half=2.0,
                   n_phi_sectors=18, pt_mode=1, pt_min=0.05),
    # the same with mean energy loss: the layer that scatters with x/X0 = 5e-4, taken as neon
    # (X0 = 28.93 g/cm^2), is 0.0145 g/cm^2 thick
    "pbpb2m_eloss": dict(BASE, n_tracks=2_000_000, xx0=5e-4, p_drop=0.05, p_outlier=0.01, outlier_half=2.0,
                         n_phi_sectors=18, pt_mode=1, pt_min=0.05, xrho=0.0145),
}


@dataclass
class Frame:
    """One SoA time frame: clusters of a track are contiguous, rows ascending."""
    offsets: np.ndarray   # int64[nt+1]
    x: np.ndarray         # float32[nc]
    y: np.ndarray
    z: np.ndarray
    sy2: np.ndarray
    sz2: np.ndarray
    row: np.ndarray       # uint8[nc]
    sector: np.ndarray    # uint8[nt]
    truth: Optional[np.ndarray] = None         # float64[nc,5] true (y,z,snp,tgl,q/pT) at each cluster
    flags: Optional[np.ndarray] = None         # uint8[nc], bit0 = outlier
    truth_vertex: Optional[np.ndarray] = None  # float64[nt,6]
    params: dict = field(default_factory=dict)

    @property
    def n_tracks(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_clusters(self) -> int:
        return int(self.offsets[-1])

    def subset(self, t0: int, t1: int) -> "Frame":
        """Tracks [t0, t1) as a new frame with rebased offsets (arrays are views)."""
        a, b = int(self.offsets[t0]), int(self.offsets[t1])
        sl = slice(a, b)
        return Frame(self.offsets[t0:t1 + 1] - a, self.x[sl], self.y[sl], self.z[sl], self.sy2[sl], self.sz2[sl],
                     self.row[sl], self.sector[t0:t1],
                     None if self.truth is None else self.truth[sl],
                     None if self.flags is None else self.flags[sl],
                     None if self.truth_vertex is None else self.truth_vertex[t0:t1], dict(self.params))


def generate(preset: str = "sector1k", seed: int = 0, truth: bool = False, threads: Optional[int] = None,
             **overrides) -> Frame:
    """Generate one frame.  ``overrides`` replace preset fields (e.g. n_tracks=...)."""
    lib = _load()
    p = dict(PRESETS[preset]) if isinstance(preset, str) else dict(preset)
    p.update(overrides)
    p.setdefault("track_id_offset", 0)
    cfg = _Config()
    for name, _ in _Config._fields_:
        if name in ("seed", "n_threads"):
            continue
        setattr(cfg, name, p[name])
    cfg.seed = seed
    cfg.n_threads = threads if threads else min(os.cpu_count() or 1, 64)
    nt = int(p["n_tracks"])
    counts = np.zeros(nt, dtype=np.int32)
    if lib.tpcgen_count(ctypes.byref(cfg), counts.ctypes.data) != 0:
        raise RuntimeError("tpcgen_count failed")
    offsets = np.zeros(nt + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    nc = int(offsets[-1])
    arr = {k: np.empty(nc, dtype=np.float32) for k in ("x", "y", "z", "sy2", "sz2")}
    row = np.empty(nc, dtype=np.uint8)
    sector = np.zeros(nt, dtype=np.uint8)
    tr = np.empty((nc, 5), dtype=np.float64) if truth else None
    fl = np.zeros(nc, dtype=np.uint8) if truth else None
    tv = np.empty((nt, 6), dtype=np.float64) if truth else None
    out = _Out()
    out.offsets = offsets.ctypes.data
    for k in arr:
        setattr(out, k, arr[k].ctypes.data)
    out.row = row.ctypes.data
    out.sector = sector.ctypes.data
    out.truth = tr.ctypes.data if tr is not None else None
    out.flags = fl.ctypes.data if fl is not None else None
    out.truth_vertex = tv.ctypes.data if tv is not None else None
    if lib.tpcgen_fill(ctypes.byref(cfg), ctypes.byref(out)) != 0:
        raise RuntimeError("tpcgen_fill failed")
    p["seed"] = seed
    return Frame(offsets, arr["x"], arr["y"], arr["z"], arr["sy2"], arr["sz2"], row, sector, tr, fl, tv, p)


def lognormal_sizes(n: int, median: float, sigma_ln: float, lo: float, hi: float, seed: int = 0) -> np.ndarray:
    """Sizes drawn log-normally (median, log width), redrawn outside [lo, hi]."""
    out = np.empty(n, dtype=np.int64)
    _load().tpcgen_lognormal_sizes(seed, n, median, sigma_ln, lo, hi, out.ctypes.data)
    return out


def event_batch(n_events: int = 4096, median: float = 800.0, sigma_ln: float = 1.0, lo: float = 10.0,
                hi: float = 20000.0, seed: int = 0, preset: str = "detector50k", threads: Optional[int] = None,
                **overrides) -> tuple:
    """Many independent events of uneven multiplicity in one frame.

    Tracks per event are log-normal (median, log width, redrawn outside
    [lo, hi]); the events' tracks are concatenated, event e holding tracks
    [event_offsets[e], event_offsets[e+1]).  Tracks are generated
    independently (keyed by seed and track index), so concatenating events
    and generating one frame of the total size give the same tracks.
    Returns (Frame, event_offsets int64[n_events+1])."""
    sizes = lognormal_sizes(n_events, median, sigma_ln, lo, hi, seed=seed + 1000003)
    ev = np.zeros(n_events + 1, dtype=np.int64)
    np.cumsum(sizes, out=ev[1:])
    f = generate(preset, seed=seed, threads=threads, n_tracks=int(ev[-1]), **overrides)
    f.params["event_sizes"] = dict(n_events=n_events, median=median, sigma_ln=sigma_ln, lo=lo, hi=hi)
    return f, ev


def poisson_arrivals(n: int, rate_hz: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    out = np.empty(n, dtype=np.float64)
    _load().tpcgen_poisson_arrivals(seed, n, rate_hz, out.ctypes.data)
    return out


def row_x_table(n_rows: int = N_ROWS, x0: float = ROW_X0, pitch: float = ROW_PITCH) -> np.ndarray:
    """Pad-row plane positions as stored in the frames (float32-rounded)."""
    return (x0 + np.arange(n_rows, dtype=np.float64) * pitch).astype(np.float32)
