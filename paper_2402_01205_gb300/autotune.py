"""Autotuner for the fit kernel's launch shape.

The persistent fit kernel has three launch choices that change its speed but
not its results (every choice is bit-identical; the GPU tests check it):

* ``block_threads``  threads per block, 128 or 256 (tracks per warp are fixed
  at 32, one track per lane: each warp-wide FP64 instruction of the
  innovation inverse and chi2 costs the FP64 pipe the same with 1 or 32
  lanes active, and about three quarters of a step (propagation scalars,
  residual, S, the FP64 island, the gain) cannot be split between lanes, so
  k lanes per track would raise both the FP64 pipe time and the issue slots
  per cluster about k-fold; two tracks per lane, advanced with paired FP32
  instructions, was built and measured 1.8 times slower on the Pb-Pb frame:
  half the resident warps, and packing the pairs cost more issue slots than
  the pairing saved);
* ``blocks_per_sm``  resident blocks per SM (grid = SMs x blocks_per_sm);
* ``sort_tracks``    longest-first order of tracks, or frame order.

``tune`` times every candidate on the caller's device frame through a
captured batch graph (CUDA events on the replay stream, median of a few
replays) and returns the fastest; ``save`` / ``load`` / ``lookup`` keep the
choices in a JSON tune table keyed by device and frame size class, and
``config_for`` turns an entry into ``Fitter`` keyword arguments.
"""
from __future__ import annotations

import json
import math
import os
import statistics
from typing import Callable, Iterable, Optional

# occupancy ceilings of the plain fit: blocks of 128 up to 5 per SM (an
# instantiation for at most 102 registers per thread), of 256 up to 2
MAX_BLOCKS_PER_SM = {128: 5, 256: 2}
TUNABLE = ("block_threads", "blocks_per_sm", "sort_tracks")


def candidates(block_threads: Iterable[int] = (128, 256), sort_tracks: Iterable[int] = (1, 0)) -> list:
    """Every launch shape the kernel can take."""
    out = []
    for bt in block_threads:
        for bps in range(1, MAX_BLOCKS_PER_SM[bt] + 1):
            for srt in sort_tracks:
                out.append({"block_threads": bt, "blocks_per_sm": bps, "sort_tracks": srt})
    return out


def size_class(n_tracks: int) -> str:
    """Frames are tuned per power-of-four track-count class."""
    return "nt4^%d" % (0 if n_tracks < 1 else int(math.log(n_tracks, 4)))


def table_key(device_name: str, sms: int, n_tracks: int) -> str:
    return f"{device_name}|{sms}SM|{size_class(n_tracks)}"


def select(timings: dict) -> tuple:
    """The fastest candidate; ties go to the earlier candidate."""
    best_key, best_ms = None, math.inf
    for key, ms in timings.items():
        if ms < best_ms:
            best_key, best_ms = key, ms
    if best_key is None:
        raise ValueError("no timings")
    return dict(best_key), best_ms


def measure_batch(T, frame, cand: dict, reps: int = 5, warmup: int = 1, device: int = 0) -> float:
    """Median device time (ms) of one replay of the batch graph under `cand`."""
    import torch
    stream = torch.cuda.Stream(device=device)
    with T.Fitter(device=device, **cand) as fx, T.Batch(fx, frame) as b:
        for _ in range(warmup):
            b.launch(stream)
        b.sync()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.launch(stream)
            e1.record(stream)
            b.sync()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def tune(T, frame, cands: Optional[list] = None, reps: int = 5, device: int = 0,
         timer: Optional[Callable] = None) -> dict:
    """Time every candidate on `frame` and return the table entry of the best.

    `timer(cand) -> ms` replaces the GPU measurement (host-logic tests)."""
    cands = cands if cands is not None else candidates()
    timer = timer or (lambda c: measure_batch(T, frame, c, reps=reps, device=device))
    timings = {}
    for c in cands:
        timings[tuple(sorted(c.items()))] = float(timer(c))
    best, ms = select(timings)
    return {"choice": best, "ms": ms,
            "all": [{**dict(k), "ms": v} for k, v in sorted(timings.items(), key=lambda kv: kv[1])]}


def load(path: str) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def save(path: str, key: str, entry: dict) -> dict:
    """Insert or replace one entry (atomic rename)."""
    table = load(path)
    table[key] = entry
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return table


def lookup(table: dict, device_name: str, sms: int, n_tracks: int) -> Optional[dict]:
    """The entry for this device and size class, else the nearest size class
    tuned on the same device, else None."""
    key = table_key(device_name, sms, n_tracks)
    if key in table:
        return table[key]
    prefix = f"{device_name}|{sms}SM|nt4^"
    same = [(int(k[len(prefix):]), v) for k, v in table.items() if k.startswith(prefix)]
    if not same:
        return None
    want = int(size_class(n_tracks)[4:])
    return min(same, key=lambda kv: (abs(kv[0] - want), kv[0]))[1]


def config_for(entry: Optional[dict]) -> dict:
    """Fitter keyword arguments of a table entry ({} = library defaults)."""
    if not entry:
        return {}
    return {k: int(entry["choice"][k]) for k in TUNABLE if k in entry["choice"]}
