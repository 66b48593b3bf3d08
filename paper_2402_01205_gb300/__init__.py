"""Batched TPC Kalman track fit on GB300: Python binding of libtpcfit (ctypes).

Argument marshalling only: every step of the fit runs in the CUDA library
(``csrc/``).  The functions mirror the C-ABI of ``include/tpcfit.h``
(``create``, ``fit``, ``fit_async``, ``sync``, ``submit``, ``poll``, ``wait``,
``destroy``); ``Fitter`` wraps a handle.  Frames are objects with ``offsets``,
``x``, ``y``, ``z``, ``sy2``, ``sz2``, ``row`` arrays: CUDA torch tensors are
passed as device memory, numpy arrays / CPU tensors as host memory.  PyTorch
provides device memory and streams only.

The library must be built (``_build.build()``); there is no fallback: a
missing library raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import _build

__all__ = ["TpcfitError", "Config", "default_config", "create", "destroy", "fit", "fit_async", "sync", "submit",
           "poll", "wait", "last_timing", "reset_timing", "probe_fma_rates", "strerror", "now", "Fitter",
           "library_path", "alloc_result", "STATUS_NAMES", "Batch", "EventViews", "batch_create", "batch_launch",
           "batch_sync", "batch_destroy", "fit_noalloc", "rans_bound", "rans_encode", "rans_decode", "FollowConfig",
           "follow_config", "follow", "gather_tracks"]

OK, E_INVAL, E_NOMEM, E_CUDA, E_TIMEOUT, E_BUSY, E_NOTFOUND, E_NODEV = 0, -1, -2, -3, -4, -5, -6, -7
MEM_HOST, MEM_DEVICE = 0, 1
PENDING, DONE, FAILED = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "TOO_FEW", 2: "SNP_LIMIT", 3: "NOT_PD", 4: "NONFINITE", 5: "BAD_INPUT", 6: "STOPPED",
                7: "DERAILED"}


class TpcfitError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tpcfit error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("bz_tesla", ctypes.c_float), ("chi2_max", ctypes.c_float), ("xx0_per_row", ctypes.c_float),
        ("mass_gev", ctypes.c_float), ("snp_max", ctypes.c_float), ("seed_cov", ctypes.c_float * 5),
        ("restart_scale", ctypes.c_float), ("min_clusters", ctypes.c_int32), ("n_rows", ctypes.c_int32),
        ("row_x0_cm", ctypes.c_float), ("row_pitch_cm", ctypes.c_float), ("hbm_budget_bytes", ctypes.c_uint64),
        ("max_slots", ctypes.c_int32), ("device", ctypes.c_int32), ("block_threads", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32), ("sort_tracks", ctypes.c_int32), ("res_step_y_cm", ctypes.c_float),
        ("res_step_z_cm", ctypes.c_float), ("xrho_per_row", ctypes.c_float), ("eloss_z_over_a", ctypes.c_float),
        ("eloss_i_ev", ctypes.c_float), ("fit_iterations", ctypes.c_int32), ("reseed_pct", ctypes.c_int32),
        ("host_chunk_clusters", ctypes.c_int64),
    ]


class _Frame(ctypes.Structure):
    _fields_ = [("n_tracks", ctypes.c_int64), ("n_clusters", ctypes.c_int64), ("track_offsets", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p), ("sy2", ctypes.c_void_p),
                ("sz2", ctypes.c_void_p), ("row", ctypes.c_void_p), ("sector", ctypes.c_void_p),
                ("mem", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_void_p), ("cov", ctypes.c_void_p), ("x_ref", ctypes.c_void_p),
                ("chi2", ctypes.c_void_p), ("ndf", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("accept", ctypes.c_void_p), ("mem", ctypes.c_int32), ("chi2_out_cluster", ctypes.c_void_p),
                ("chi2_in_cluster", ctypes.c_void_p), ("restart_state", ctypes.c_void_p), ("res_y", ctypes.c_void_p),
                ("res_z", ctypes.c_void_p), ("smoothed_state", ctypes.c_void_p), ("smoothed_cov", ctypes.c_void_p)]


class _ServeStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("parts", ctypes.c_int64), ("max_parts_per_launch", ctypes.c_int64)]


class _Timing(ctypes.Structure):
    _fields_ = [("prepare_ms", ctypes.c_float), ("sort_ms", ctypes.c_float), ("fit_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float), ("kernel_launches", ctypes.c_int32), ("fit_grid", ctypes.c_int32),
                ("fit_block", ctypes.c_int32), ("fit_regs", ctypes.c_int32), ("n_timed", ctypes.c_int64),
                ("prepare_ms_sum", ctypes.c_double), ("sort_ms_sum", ctypes.c_double),
                ("fit_ms_sum", ctypes.c_double), ("total_ms_sum", ctypes.c_double)]


class FollowConfig(ctypes.Structure):
    _fields_ = [("window_sigma", ctypes.c_float), ("nominal_v", ctypes.c_float), ("max_miss", ctypes.c_int32),
                ("tan_edge", ctypes.c_float), ("z_max", ctypes.c_float), ("seed_cov", ctypes.c_float * 5),
                ("n_sectors", ctypes.c_int32), ("n_ybins", ctypes.c_int32), ("n_zbins", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class _Hits(ctypes.Structure):
    _fields_ = [("n_clusters", ctypes.c_int64)] + [(k, ctypes.c_void_p) for k in
                                                    ("x", "y", "z", "sy2", "sz2", "row", "sector")]


class _Seeds(ctypes.Structure):
    _fields_ = [("n_seeds", ctypes.c_int64), ("state", ctypes.c_void_p), ("row", ctypes.c_void_p),
                ("sector", ctypes.c_void_p)]


class _Tracks(ctypes.Structure):
    _fields_ = [("att", ctypes.c_void_p), ("n_att", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("state", ctypes.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libtpcfit.so is not built ({_build.LIB}); run paper_2402_01205_gb300._build.build()")
    lib = ctypes.CDLL(_build.LIB)
    H = ctypes.c_void_p
    lib.tpcfit_default_config.argtypes = [ctypes.POINTER(Config)]
    lib.tpcfit_default_config.restype = None
    lib.tpcfit_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(H)]
    lib.tpcfit_fit.argtypes = [H, ctypes.POINTER(_Frame), ctypes.POINTER(_Result)]
    lib.tpcfit_fit_async.argtypes = [H, ctypes.POINTER(_Frame), ctypes.POINTER(_Result), ctypes.c_void_p]
    lib.tpcfit_sync.argtypes = [H, ctypes.c_double]
    lib.tpcfit_submit.argtypes = [H, ctypes.POINTER(_Frame), ctypes.POINTER(_Result), ctypes.POINTER(ctypes.c_uint64)]
    lib.tpcfit_poll.argtypes = [H, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.tpcfit_wait.argtypes = [H, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_double)]
    lib.tpcfit_last_timing.argtypes = [H, ctypes.POINTER(_Timing)]
    lib.tpcfit_get_serve_stats.argtypes = [H, ctypes.POINTER(_ServeStats)]
    lib.tpcfit_reset_timing.argtypes = [H]
    lib.tpcfit_probe_fma_rates.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    lib.tpcfit_destroy.argtypes = [H]
    lib.tpcfit_strerror.argtypes = [ctypes.c_int]
    lib.tpcfit_strerror.restype = ctypes.c_char_p
    lib.tpcfit_last_error_message.argtypes = []
    lib.tpcfit_last_error_message.restype = ctypes.c_char_p
    lib.tpcfit_now.argtypes = []
    lib.tpcfit_now.restype = ctypes.c_double
    lib.tpcfit_rans_bound.argtypes = [ctypes.c_int64, ctypes.c_int32]
    lib.tpcfit_rans_bound.restype = ctypes.c_int64
    lib.tpcfit_rans_encode.argtypes = [H, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    lib.tpcfit_rans_decode.argtypes = [H, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_void_p]
    lib.tpcfit_fit_noalloc.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(_Frame), ctypes.POINTER(_Result),
                                       ctypes.c_void_p]
    lib.tpcfit_fit_noalloc.restype = ctypes.c_int
    lib.tpcfit_follow_default_config.argtypes = [ctypes.POINTER(FollowConfig)]
    lib.tpcfit_follow_default_config.restype = None
    lib.tpcfit_follow.argtypes = [H, ctypes.POINTER(FollowConfig), ctypes.POINTER(_Hits), ctypes.POINTER(_Seeds),
                                  ctypes.POINTER(_Tracks), ctypes.c_void_p]
    lib.tpcfit_follow.restype = ctypes.c_int
    lib.tpcfit_gather_tracks.argtypes = [H, ctypes.POINTER(_Hits), ctypes.POINTER(_Tracks), ctypes.c_int64] + \
        [ctypes.c_void_p] * 7 + [ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    lib.tpcfit_gather_tracks.restype = ctypes.c_int
    lib.tpcfit_batch_create.argtypes = [H, ctypes.POINTER(_Frame), ctypes.POINTER(_Result), ctypes.POINTER(H)]
    lib.tpcfit_batch_launch.argtypes = [H, ctypes.c_void_p]
    lib.tpcfit_batch_sync.argtypes = [H, ctypes.c_double]
    lib.tpcfit_batch_destroy.argtypes = [H]
    for fn in ("tpcfit_create", "tpcfit_fit", "tpcfit_fit_async", "tpcfit_sync", "tpcfit_submit", "tpcfit_poll",
               "tpcfit_wait", "tpcfit_last_timing", "tpcfit_reset_timing", "tpcfit_destroy", "tpcfit_get_serve_stats",
               "tpcfit_probe_fma_rates", "tpcfit_batch_create", "tpcfit_batch_launch", "tpcfit_batch_sync",
               "tpcfit_batch_destroy", "tpcfit_rans_encode", "tpcfit_rans_decode"):
        getattr(lib, fn).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int) -> int:
    if rc < 0:
        lib = _load()
        raise TpcfitError(rc, f"{lib.tpcfit_strerror(rc).decode()}: {lib.tpcfit_last_error_message().decode()}")
    return rc


def strerror(code: int) -> str:
    return _load().tpcfit_strerror(code).decode()


def now() -> float:
    return _load().tpcfit_now()


def default_config(**overrides) -> Config:
    cfg = Config()
    _load().tpcfit_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "seed_cov":
            cfg.seed_cov = (ctypes.c_float * 5)(*v)
        else:
            setattr(cfg, k, v)
    return cfg


# ---------------------------------------------------------------- marshalling
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a) -> int:
    if a is None:
        return 0
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays must be C-contiguous")
    return a.ctypes.data


_DT = {"offsets": "int64", "x": "float32", "y": "float32", "z": "float32", "sy2": "float32", "sz2": "float32",
       "row": "uint8"}


def _mem_of(arrs) -> int:
    dev = [_is_torch(a) and a.is_cuda for a in arrs]
    if all(dev):
        return MEM_DEVICE
    if not any(dev):
        return MEM_HOST
    raise ValueError("frame arrays must all be on the GPU or all on the host")


def _check_dtypes(obj, names):
    for k in names:
        a = getattr(obj, k)
        dt = str(a.dtype).replace("torch.", "")
        if dt != _DT.get(k, dt):
            raise TypeError(f"{k} must be {_DT[k]}, got {dt}")


def _frame_struct(frame) -> tuple:
    """The C frame of `frame`; a host frame may have x = None (clusters on
    their pad-row planes: the library derives x from the rows)."""
    names = ("offsets", "x", "y", "z", "sy2", "sz2", "row")
    present = tuple(k for k in names if getattr(frame, k, None) is not None)
    if set(names) - set(present) - {"x"}:
        raise ValueError(f"frame lacks {sorted(set(names) - set(present) - {'x'})}")
    arrs = [getattr(frame, k) for k in present]
    _check_dtypes(frame, present)
    mem = _mem_of(arrs)
    if "x" not in present and mem != MEM_HOST:
        raise ValueError("x may be None only in a host frame")
    nt = int(frame.offsets.shape[0]) - 1
    nc = int(frame.y.shape[0])
    for k in present[1:]:
        if int(getattr(frame, k).shape[0]) != nc:
            raise ValueError(f"{k} has {getattr(frame, k).shape[0]} entries, y has {nc}")
    ptr = {k: _ptr(getattr(frame, k)) for k in present}
    f = _Frame(nt, nc, ptr["offsets"], ptr.get("x"), ptr["y"], ptr["z"], ptr["sy2"], ptr["sz2"], ptr["row"], 0, mem)
    return f, mem, nt, nc


def alloc_result(n_tracks: int, n_clusters: int, device=None, pinned: bool = False, residuals: bool = False,
                 smoothed: bool = False) -> dict:
    """Result buffers: torch tensors on ``device`` (CUDA) or numpy arrays on the
    host (pinned torch tensors with ``pinned``).  ``residuals`` adds the int16
    track-model compression residual codes ``res_y``, ``res_z``; ``smoothed``
    the two-filter smoother's per-cluster ``smoothed_state`` (n_clusters, 5)
    and ``smoothed_cov`` (n_clusters, 15), which select the smoother."""
    if device is not None or pinned:
        import torch
        kw = dict(device=device) if device is not None else dict(pin_memory=True)
        mk = lambda shape, dt: torch.empty(shape, dtype=dt, **kw)  # noqa: E731
        out = dict(state=mk((n_tracks, 5), torch.float32), cov=mk((n_tracks, 15), torch.float32),
                   x_ref=mk((n_tracks,), torch.float32), chi2=mk((n_tracks,), torch.float64),
                   ndf=mk((n_tracks,), torch.int32), status=mk((n_tracks,), torch.int32),
                   accept=mk((n_clusters,), torch.uint8))
        if residuals:
            out.update(res_y=mk((n_clusters,), torch.int16), res_z=mk((n_clusters,), torch.int16))
        if smoothed:
            out.update(smoothed_state=mk((n_clusters, 5), torch.float32), smoothed_cov=mk((n_clusters, 15), torch.float32))
        return out
    out = dict(state=np.empty((n_tracks, 5), np.float32), cov=np.empty((n_tracks, 15), np.float32),
               x_ref=np.empty(n_tracks, np.float32), chi2=np.empty(n_tracks, np.float64),
               ndf=np.empty(n_tracks, np.int32), status=np.empty(n_tracks, np.int32),
               accept=np.empty(n_clusters, np.uint8))
    if residuals:
        out.update(res_y=np.empty(n_clusters, np.int16), res_z=np.empty(n_clusters, np.int16))
    if smoothed:
        out.update(smoothed_state=np.empty((n_clusters, 5), np.float32),
                   smoothed_cov=np.empty((n_clusters, 15), np.float32))
    return out


# Elements per track (or per cluster) of each result array.
_RES_TRACK = {"state": 5, "cov": 15, "x_ref": 1, "chi2": 1, "ndf": 1, "status": 1, "restart_state": 5}
_RES_CLUSTER = {"accept": 1, "res_y": 1, "res_z": 1, "chi2_out_cluster": 1, "chi2_in_cluster": 1, "smoothed_state": 5,
                "smoothed_cov": 15}


def _numel(a) -> int:
    return int(a.numel()) if _is_torch(a) else int(a.size)


def _result_struct(res: dict, nt: int, nc: int) -> tuple:
    """The C result of `res` for a frame of nt tracks and nc clusters: every
    buffer must hold exactly its frame's number of elements (a result of
    another frame would be written past its end)."""
    names = ("state", "cov", "x_ref", "chi2", "ndf", "status", "accept")
    arrs = [res[k] for k in names]
    mem = _mem_of(arrs)
    for k, a in res.items():
        if a is None or (k not in _RES_TRACK and k not in _RES_CLUSTER):
            continue
        want = _RES_TRACK[k] * nt if k in _RES_TRACK else _RES_CLUSTER[k] * nc
        if _numel(a) != want:
            raise ValueError(f"result {k} has {_numel(a)} elements, the frame needs {want}")
    extra = [_ptr(res.get(k)) for k in ("chi2_out_cluster", "chi2_in_cluster", "restart_state", "res_y", "res_z",
                                         "smoothed_state", "smoothed_cov")]
    for k in ("res_y", "res_z"):
        if res.get(k) is not None:
            dt = str(res[k].dtype).replace("torch.", "")
            if dt != "int16":
                raise TypeError(f"{k} must be int16, got {dt}")
    return _Result(*[_ptr(a) for a in arrs], mem, *extra), mem


# ---------------------------------------------------------------- C-ABI mirror
def create(config: Optional[Config] = None) -> int:
    lib = _load()
    h = ctypes.c_void_p()
    _check(lib.tpcfit_create(ctypes.byref(config) if config is not None else None, ctypes.byref(h)))
    return h.value


def destroy(handle: int) -> None:
    _check(_load().tpcfit_destroy(handle))


def fit(handle: int, frame, res: dict) -> dict:
    f, _, nt, nc = _frame_struct(frame)
    r, _ = _result_struct(res, nt, nc)
    _check(_load().tpcfit_fit(handle, ctypes.byref(f), ctypes.byref(r)))
    return res


def fit_async(handle: int, frame, res: dict, stream=None) -> dict:
    """Enqueue on a torch.cuda.Stream (or raw cudaStream_t int, or None)."""
    f, _, nt, nc = _frame_struct(frame)
    r, _ = _result_struct(res, nt, nc)
    s = getattr(stream, "cuda_stream", stream)
    _check(_load().tpcfit_fit_async(handle, ctypes.byref(f), ctypes.byref(r), s))
    return res


def sync(handle: int, timeout_s: float = -1.0) -> None:
    _check(_load().tpcfit_sync(handle, timeout_s))


def submit(handle: int, frame, res: dict) -> int:
    f, _, nt, nc = _frame_struct(frame)
    r, _ = _result_struct(res, nt, nc)
    t = ctypes.c_uint64()
    _check(_load().tpcfit_submit(handle, ctypes.byref(f), ctypes.byref(r), ctypes.byref(t)))
    return t.value


def poll(handle: int, ticket: int) -> tuple:
    st, td = ctypes.c_int(), ctypes.c_double()
    _check(_load().tpcfit_poll(handle, ticket, ctypes.byref(st), ctypes.byref(td)))
    return st.value, td.value


def wait(handle: int, ticket: int, timeout_s: float = -1.0) -> tuple:
    st, td = ctypes.c_int(), ctypes.c_double()
    _check(_load().tpcfit_wait(handle, ticket, timeout_s, ctypes.byref(st), ctypes.byref(td)))
    return st.value, td.value


def serve_stats(handle: int) -> dict:
    s = _ServeStats()
    _check(_load().tpcfit_get_serve_stats(handle, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in _ServeStats._fields_}


def last_timing(handle: int) -> dict:
    t = _Timing()
    _check(_load().tpcfit_last_timing(handle, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in _Timing._fields_}


def reset_timing(handle: int) -> None:
    _check(_load().tpcfit_reset_timing(handle))


def probe_fma_rates(device: int = 0) -> dict:
    """Measured FP64 / FP32 FMA lane-operations per second and the SM clock (kHz)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(_load().tpcfit_probe_fma_rates(device, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return dict(fp64_fma_per_s=a.value, fp32_fma_per_s=b.value, sm_clock_khz=c.value)


def fit_noalloc(frame, res: dict, config: Optional[Config] = None, stream=None) -> dict:
    """tpcfit_fit_noalloc: fit a device frame without allocating device memory.

    For callers that cannot allocate while they run (their device memory is
    owned by another allocator, or their steady-state loop forbids
    allocation).  Scratch comes from a static device array sized for
    TPCFIT_NOALLOC_MAX_TRACKS (65536) tracks, shared by all calls: calls must
    not overlap on the GPU.  Blocks until the fit is done."""
    lib = _load()
    fn = lib.tpcfit_fit_noalloc
    fn.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(_Frame), ctypes.POINTER(_Result), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    f, _, nt, nc = _frame_struct(frame)
    r, _ = _result_struct(res, nt, nc)
    s = getattr(stream, "cuda_stream", stream)
    _check(fn(ctypes.byref(config) if config is not None else None, ctypes.byref(f), ctypes.byref(r), s))
    return res


def batch_create(handle: int, frame, res: dict) -> int:
    f, _, nt, nc = _frame_struct(frame)
    r, _ = _result_struct(res, nt, nc)
    b = ctypes.c_void_p()
    _check(_load().tpcfit_batch_create(handle, ctypes.byref(f), ctypes.byref(r), ctypes.byref(b)))
    return b.value


def batch_launch(batch: int, stream=None) -> None:
    _check(_load().tpcfit_batch_launch(batch, getattr(stream, "cuda_stream", stream)))


def batch_sync(batch: int, timeout_s: float = -1.0) -> None:
    _check(_load().tpcfit_batch_sync(batch, timeout_s))


def batch_destroy(batch: int) -> None:
    _check(_load().tpcfit_batch_destroy(batch))


def rans_bound(n: int, segment_symbols: int = 0) -> int:
    """Largest rANS container size (bytes) for n codes."""
    b = _load().tpcfit_rans_bound(n, segment_symbols)
    if b < 0:
        raise TpcfitError(E_INVAL, "bad rANS sizes")
    return b


def rans_encode(handle: int, codes, segment_symbols: int = 0, out=None, stream=None):
    """Entropy-code a CUDA int16 tensor; returns (uint8 CUDA tensor, container bytes)."""
    import torch
    if not (_is_torch(codes) and codes.is_cuda and codes.dtype == torch.int16 and codes.is_contiguous()):
        raise TypeError("codes must be a contiguous CUDA int16 tensor")
    n = int(codes.numel())
    if out is None:
        out = torch.empty(rans_bound(n, segment_symbols), dtype=torch.uint8, device=codes.device)
    size = ctypes.c_int64()
    _check(_load().tpcfit_rans_encode(handle, codes.data_ptr() if n else None, n, segment_symbols, out.data_ptr(),
                                      out.numel(), ctypes.byref(size), getattr(stream, "cuda_stream", stream)))
    return out, size.value


def rans_decode(handle: int, blob, size: int, n: int, out=None, stream=None):
    """Decode a container held in a CUDA uint8 tensor into n int16 codes (CUDA tensor)."""
    import torch
    if out is None:
        out = torch.empty(n, dtype=torch.int16, device=blob.device)
    _check(_load().tpcfit_rans_decode(handle, blob.data_ptr(), size, out.data_ptr() if n else None, n,
                                      getattr(stream, "cuda_stream", stream)))
    return out


def follow_config(**overrides) -> FollowConfig:
    c = FollowConfig()
    _load().tpcfit_follow_default_config(ctypes.byref(c))
    for k, v in overrides.items():
        if k == "seed_cov":
            c.seed_cov = (ctypes.c_float * 5)(*v)
        else:
            setattr(c, k, v)
    return c


def _dev(a, dtype: str, name: str):
    import torch
    if not (_is_torch(a) and a.is_cuda and a.is_contiguous() and str(a.dtype) == "torch." + dtype):
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return a.data_ptr()


def _hits_struct(hits) -> _Hits:
    """hits: object with CUDA tensors x, y, z, sy2, sz2 (float32), row and sectors (uint8), one per cluster."""
    n = int(hits.y.numel())
    return _Hits(n, *[_dev(getattr(hits, k), "float32", k) for k in ("x", "y", "z", "sy2", "sz2")],
                 _dev(hits.row, "uint8", "row"), _dev(hits.sectors, "uint8", "sectors"))


def follow(handle: int, hits, seeds: dict, config: Optional[FollowConfig] = None, stream=None,
           n_rows: int = 152) -> dict:
    """Track following (tpcfit_follow): seeds dict of CUDA tensors state (float32 [ns, 5]),
    row and sector (uint8 [ns]); returns CUDA tensors att [ns, n_rows], n_att, status, state."""
    import torch
    h = _hits_struct(hits)
    ns = int(seeds["state"].shape[0])
    sd = _Seeds(ns, _dev(seeds["state"], "float32", "state"), _dev(seeds["row"], "uint8", "row"),
                _dev(seeds["sector"], "uint8", "sector"))
    dev = seeds["state"].device
    lib = _load()
    out = dict(att=torch.empty((ns, n_rows), dtype=torch.int32, device=dev),
               n_att=torch.empty(ns, dtype=torch.int32, device=dev), status=torch.empty(ns, dtype=torch.int32, device=dev),
               state=torch.empty((ns, 5), dtype=torch.float32, device=dev))
    tr = _Tracks(out["att"].data_ptr(), out["n_att"].data_ptr(), out["status"].data_ptr(), out["state"].data_ptr())
    _check(lib.tpcfit_follow(handle, ctypes.byref(config) if config is not None else None, ctypes.byref(h),
                             ctypes.byref(sd), ctypes.byref(tr), getattr(stream, "cuda_stream", stream)))
    out["_keep"] = (hits, seeds)
    return out


def gather_tracks(handle: int, hits, tracks: dict, stream=None):
    """tpcfit_gather_tracks: the followed tracks as a device frame (SimpleNamespace of CUDA tensors)."""
    import types
    import torch
    h = _hits_struct(hits)
    ns = int(tracks["n_att"].numel())
    dev = tracks["n_att"].device
    # the follow results are complete once the stream they were produced on is
    if stream is None:
        sync(handle)
    else:
        stream.synchronize()
    cap = int(tracks["n_att"].sum().item())
    fr = types.SimpleNamespace(offsets=torch.empty(ns + 1, dtype=torch.int64, device=dev),
                               **{k: torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
                                  for k in ("x", "y", "z", "sy2", "sz2")},
                               row=torch.empty(max(cap, 1), dtype=torch.uint8, device=dev))
    tr = _Tracks(tracks["att"].data_ptr(), tracks["n_att"].data_ptr(), tracks["status"].data_ptr(), 0)
    n = ctypes.c_int64()
    _check(_load().tpcfit_gather_tracks(handle, ctypes.byref(h), ctypes.byref(tr), ns, fr.offsets.data_ptr(),
                                        *[getattr(fr, k).data_ptr() for k in ("x", "y", "z", "sy2", "sz2", "row")],
                                        max(cap, 1), ctypes.byref(n), getattr(stream, "cuda_stream", stream)))
    for k in ("x", "y", "z", "sy2", "sz2", "row"):
        setattr(fr, k, getattr(fr, k)[:n.value])
    return fr


class EventViews:
    """Per-event frames and results inside one concatenated device frame.

    For fitting the events of a batch one plain launch sequence per event:
    event e's frame points into the concatenated cluster arrays and result
    buffers, with its own offsets rebased to 0 (kept in one device tensor)."""

    def __init__(self, frame, res: dict, event_offsets):
        import torch
        ev = np.asarray(event_offsets, dtype=np.int64)
        off = frame.offsets.cpu().numpy() if _is_torch(frame.offsets) else np.asarray(frame.offsets)
        ne = len(ev) - 1
        reb = np.empty(int(ev[-1]) + ne, dtype=np.int64)
        for e in range(ne):
            t0, t1 = int(ev[e]), int(ev[e + 1])
            reb[t0 + e:t1 + e + 1] = off[t0:t1 + 1] - off[t0]
        self.rebased = torch.from_numpy(reb).to(frame.x.device)
        self.frame, self.res = frame, res
        fs, _, nt, nc = _frame_struct(frame)
        rs, _ = _result_struct(res, nt, nc)
        if fs.mem != MEM_DEVICE or rs.mem != MEM_DEVICE:
            raise ValueError("EventViews takes a device frame and device results")
        self.frames, self.results = [], []
        rb = self.rebased.data_ptr()
        for e in range(ne):
            t0, t1 = int(ev[e]), int(ev[e + 1])
            c0, c1 = int(off[t0]), int(off[t1])
            self.frames.append(_Frame(t1 - t0, c1 - c0, rb + 8 * (t0 + e), fs.x + 4 * c0, fs.y + 4 * c0,
                                      fs.z + 4 * c0, fs.sy2 + 4 * c0, fs.sz2 + 4 * c0, fs.row + c0, 0, MEM_DEVICE))
            self.results.append(_Result(rs.state + 20 * t0, rs.cov + 60 * t0, rs.x_ref + 4 * t0, rs.chi2 + 8 * t0,
                                        rs.ndf + 4 * t0, rs.status + 4 * t0, rs.accept + c0, MEM_DEVICE, 0, 0, 0,
                                        rs.res_y + 2 * c0 if rs.res_y else 0, rs.res_z + 2 * c0 if rs.res_z else 0))

    def __len__(self) -> int:
        return len(self.frames)

    def fit_async(self, fitter: "Fitter", stream=None) -> None:
        """One plain launch sequence per event, enqueued in event order on `stream`."""
        lib = _load()
        s = getattr(stream, "cuda_stream", stream)
        fn, h = lib.tpcfit_fit_async, fitter.handle
        for f, r in zip(self.frames, self.results):
            rc = fn(h, ctypes.byref(f), ctypes.byref(r), s)
            if rc < 0:
                _check(rc)


class Batch:
    """A captured launch sequence over one device frame of concatenated events.

    Keeps the frame and result tensors alive for as long as the graph may
    replay (the graph holds their device addresses)."""

    def __init__(self, fitter: "Fitter", frame, res: Optional[dict] = None):
        f, mem, nt, nc = _frame_struct(frame)
        if res is None:
            res = alloc_result(nt, nc, device=frame.x.device)
        self.frame, self.res, self._fitter = frame, res, fitter
        self.batch = batch_create(fitter.handle, frame, res)

    def launch(self, stream=None) -> dict:
        batch_launch(self.batch, stream)
        return self.res

    def sync(self, timeout_s: float = -1.0) -> None:
        batch_sync(self.batch, timeout_s)

    def close(self) -> None:
        if self.batch:
            batch_destroy(self.batch)
            self.batch = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Fitter:
    """Owns one library handle."""

    def __init__(self, config: Optional[Config] = None, **overrides):
        if config is None:
            config = default_config(**overrides)
        self.config = config
        self.handle = create(config)
        self._inflight = {}  # ticket -> (frame, result): buffers must outlive the ticket

    def fit(self, frame, res: Optional[dict] = None) -> dict:
        f, mem, nt, nc = _frame_struct(frame)
        if res is None:
            res = alloc_result(nt, nc, device=frame.x.device if mem == MEM_DEVICE else None)
        return fit(self.handle, frame, res)

    def fit_async(self, frame, res: dict, stream=None) -> dict:
        return fit_async(self.handle, frame, res, stream)

    def sync(self, timeout_s: float = -1.0) -> None:
        sync(self.handle, timeout_s)

    def submit(self, frame, res: dict) -> int:
        t = submit(self.handle, frame, res)
        self._inflight[t] = (frame, res)
        return t

    def poll(self, ticket: int) -> tuple:
        st = poll(self.handle, ticket)
        if st[0] != PENDING:
            self._inflight.pop(ticket, None)
        return st

    def wait(self, ticket: int, timeout_s: float = -1.0) -> tuple:
        st = wait(self.handle, ticket, timeout_s)
        if st[0] != PENDING:
            self._inflight.pop(ticket, None)
        return st

    def timing(self) -> dict:
        return last_timing(self.handle)

    def serve_stats(self) -> dict:
        """Serving engine counters: launches, parts fitted, most parts in one launch."""
        return serve_stats(self.handle)

    def follow(self, hits, seeds: dict, config: Optional[FollowConfig] = None, stream=None) -> dict:
        return follow(self.handle, hits, seeds, config, stream, n_rows=self.config.n_rows)

    def gather_tracks(self, hits, tracks: dict, stream=None):
        return gather_tracks(self.handle, hits, tracks, stream)

    def rans_encode(self, codes, segment_symbols: int = 0, out=None, stream=None):
        return rans_encode(self.handle, codes, segment_symbols, out, stream)

    def rans_decode(self, blob, size: int, n: int, out=None, stream=None):
        return rans_decode(self.handle, blob, size, n, out, stream)

    def reset_timing(self) -> None:
        reset_timing(self.handle)

    def close(self) -> None:
        if self.handle:
            destroy(self.handle)  # waits for every ticket
            self.handle = None
            self._inflight.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
