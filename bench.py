#!/usr/bin/env python
"""Benchmark of the batched TPC Kalman track fit on GB300.

One step = one pass of the whole hot path (offset/input checks, 3-point seeds,
longest-first sort, outward + inward Kalman passes, outputs) over one
Pb-Pb-scale synthetic time frame: 2,000,000 tracks, ~192 M clusters (seed 0,
exponential pT spectrum with mean 0.6 GeV/c, scattering, 5 % dropout, 1 %
outliers).  The frame (4.2 GB of cluster SoA) is larger than the 129 MB L2, so
no flush is needed between steps.

Prints one JSON line: clusters/s with the frame resident in HBM (``value``),
clusters/s through the C-ABI with pinned host buffers including the copies
(``e2e``), the fit kernel's roofline fraction, and the FP64 oracle timed on a
bounded sample of the same frame on the host cores (``cpu_baseline``).

``--impl reference`` times the FP64 oracle (the reference arm of this
project) on the host cores on bounded samples of the same workload.
Multi-GPU (torchrun): every rank fits its own frame (independent time frames,
no data exchange), max time over ranks, weak scaling.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from contextlib import contextmanager

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import tpcgen  # noqa: E402

WORKLOADS = {"pbpb2m": "Pb-Pb-scale time frame: 2,000,000 tracks, exponential pT (mean 0.6 GeV/c), 36 sectors, "
                       "x/X0 5e-4 per row, 5% dropout, 1% outliers, seed 0",
             "events4096": "4,096 independent events, tracks per event log-normal (median 800, sigma_ln 1.0, "
                           "10-20,000), tracks of 10-152 rows, pT log-uniform 0.2-10 GeV/c, 36 sectors, x/X0 5e-4 "
                           "per row, 5% dropout, 1% outliers, seed 0; one graph-captured persistent launch sequence "
                           "per step vs one plain launch sequence per event",
             "tracking": "track following + gather + fit of a 50,000-track frame of the 36-sector detector "
                         "(x/X0 5e-4 per row, 5% dropout, 1% outliers, seed 0); seeds: the true state at each "
                         "track's first cluster smeared by 0.3 of the seed sigma (seeded)",
             "pbpb2m_eloss": "the Pb-Pb-scale frame with mean energy loss (Bethe, neon, 0.0145 g/cm^2 per row, the "
                             "layer of x/X0 5e-4) in the generator and in the fit (its energy-loss kernel); pions",
             "serving": "time frames arriving as a Poisson process at 50 frames/s, clusters per frame log-normal "
                        "(median 20 M, sigma_ln 0.6, 1-120 M), tracks as in the 36-sector detector workload; a pool "
                        "of 64 frames (windows of one pre-generated 1.1 M-track frame) replayed on a seeded "
                        "arrival schedule; 120 GB HBM budget, 8 slots"}
# fit parameters of a workload beyond the defaults (library / oracle names)
FIT_PARAMS = {"pbpb2m_eloss": ({"xrho_per_row": 0.0145}, {"xrho": 0.0145})}
# the metric of the benchmark, the same string in both arms
METRIC = "clusters/s and tracks/s fitted on 1 GB300 at stated FP64-oracle error; p50/p99 frame latency"
FP64_PER_CLUSTER = 11         # the FP64 island as the method states it, per cluster: 4 (outward det, gate) + 7 (inward det, reciprocal, chi2, sum)
FP64_EXECUTED_PER_CLUSTER = 8 # FP64 lane-instructions the kernel executes per cluster (ncu): 2 (outward det) + 6 (inward)
BYTES_PER_CLUSTER = 22        # 21 B read (x, y, z, sy2, sz2 f32 + row u8) + 1 B accept written
BYTES_PER_TRACK = 108         # 8 B offset + 100 B results


@contextmanager
def host_timed():
    """A host-timed region: Python's garbage collector off, as timeit does, so
    that a collection of the interpreter's objects does not land inside a
    timed step (the library's own work is unaffected)."""
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks", suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


def kernel_source_hash() -> str:
    """Hash of the sources the fit kernel is compiled from (its file, the shared device code and the staging)."""
    h = hashlib.sha256()
    for name in ("fit_kernels.cu", "fit_device.cuh", "stage_device.cuh"):
        with open(os.path.join(ROOT, "paper_2402_01205_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


ISSUE_PER_SM_CLK = 4          # warp instructions issued per SM per clock (4 schedulers, one each)


def profiled_counters(n_clusters: int, launch: tuple, variant: str = ""):
    """ncu counters of one fit-kernel launch from the committed record
    (profiles/fit_kernel_counters.json): DRAM bytes and warp instructions,
    for this frame when it is the captured one, else scaled by clusters for a
    frame of the same launch shape; None for another shape or when the kernel
    source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "fit_kernel_counters.json")
    if not os.path.exists(p):
        return None, "no ncu record"
    with open(p) as fh:
        d = json.load(fh)
    if variant:
        if variant not in d.get("variants", {}):
            return None, f"no ncu record of the {variant} variant"
        d = dict(d["variants"][variant], kernel_sha256_16=d.get("kernel_sha256_16"))
    if d.get("kernel_sha256_16") != kernel_source_hash():
        return None, "kernel changed since the ncu capture"
    if tuple(launch) != tuple(d.get("launch", (0, 0))):
        return None, "no ncu capture of this launch shape (L2 reuse, hence traffic, depends on it)"
    f = n_clusters / d["n_clusters"]
    note = ("ncu capture of this launch: " if n_clusters == d["n_clusters"] else
            f"scaled by clusters from the ncu capture of {d['workload']}: ") + d["capture"]
    out = {"dram_bytes": d["dram_bytes_per_launch"] * f, "warp_inst": d["warp_inst_per_launch"] * f,
           "thread_inst": d["thread_inst_per_launch"] * f}
    if "fp32_flop_per_cluster" in d:
        out["fp32_flop_per_cluster"] = d["fp32_flop_per_cluster"]
    return out, note


FP64_NOMINAL_OPS = 0.625e12  # GB300 nominal FP64 rate (1.25 TFLOP/s), as FP64 lane-ops (an FMA counts once) per s


def fit_roofline(nc, nt, nc_fit, fit_s, launch, probe, sms, sm_mhz, variant: str = "", passes: int = 1):
    """Roofline of the fit kernel against its binding algorithmic roof.

    The fit's algorithmic work per cluster is 11 FP64 lane-operations (the
    FP64 island as the method states it: in the outward update the
    innovation-matrix determinant and the gate, in the inward update the
    determinant, the reciprocal, chi2 and its sum; a lane-operation = one
    lane of one FP64 instruction, an FMA counting once), about 800 FP32
    flops, and 22 bytes of HBM traffic (+108 per track).  On GB300 the FP64
    roof binds.  So ``achieved`` = FP64 lane-ops per launch / mean launch
    time, ``peak`` = the FP64 FMA rate measured live in the same run (one
    lane-op per FMA), and beside it the FP64 pipe's own share (the kernel
    executes 8 of the 11 on the FP64 pipe: the outward gate is decided in
    binary32 with the FP64 outcome, and the inward reciprocal and chi2 take
    3 instead of 4), the FP32 and HBM fractions and the instruction-issue
    roof (from the ncu counters committed for this kernel and launch)."""
    peaks, peak_src = measured_peaks()
    c, note = profiled_counters(nc, launch, variant)
    fp64 = FP64_PER_CLUSTER * passes * nc_fit / fit_s  # each seed iteration repeats both passes
    hbm = (BYTES_PER_CLUSTER * nc + BYTES_PER_TRACK * nt) / fit_s / 1e9
    beside = {
        "fp64_pipe": {"executed_lane_ops_per_cluster": FP64_EXECUTED_PER_CLUSTER,
                      "frac": FP64_EXECUTED_PER_CLUSTER * passes * nc_fit / fit_s / probe["fp64_fma_per_s"]},
        "hbm": {"achieved_gbs": hbm, "peak_gbs": peaks["hbm_gbs"], "frac": hbm / peaks["hbm_gbs"],
                "peak_source": peak_src, "bytes_per_cluster": BYTES_PER_CLUSTER, "bytes_per_track": BYTES_PER_TRACK},
    }
    if c and "fp32_flop_per_cluster" in c:
        f32 = c["fp32_flop_per_cluster"] * passes * nc_fit / fit_s
        beside["fp32"] = {"achieved_tflops": f32 / 1e12, "peak_tflops": 2 * probe["fp32_fma_per_s"] / 1e12,
                          "frac": f32 / (2 * probe["fp32_fma_per_s"]), "flop_per_cluster": c["fp32_flop_per_cluster"],
                          "peak_source": "2 x measured live FP32 FMA chain probe"}
    if c:
        issue_peak = ISSUE_PER_SM_CLK * sms * (sm_mhz or 2070.0) * 1e6
        ach = c["warp_inst"] / fit_s
        beside["issue"] = {"achieved_ginst_s": ach / 1e9, "peak_ginst_s": issue_peak / 1e9, "frac": ach / issue_peak,
                           "peak_source": f"{ISSUE_PER_SM_CLK} issue slots per SM per clock x {sms} SMs x sampled "
                                          "SM clock", "warp_inst_per_cluster": c["warp_inst"] / nc,
                           "active_lanes_per_inst": c["thread_inst"] / c["warp_inst"]}
    roof = {"bound": "alu", "kernel": "k_fit", "unit": "T FP64 lane-ops/s",
            "achieved": fp64 / 1e12, "peak": probe["fp64_fma_per_s"] / 1e12, "frac": fp64 / probe["fp64_fma_per_s"],
            "binding": "fp64", "lane_ops_per_cluster": FP64_PER_CLUSTER,
            "peak_source": "measured live in this run: FP64 FMA chain probe (tpcfit_probe_fma_rates); the "
                           "driver-measured peaks hold no FP64 figure",
            "frac_of_nominal": fp64 / FP64_NOMINAL_OPS,
            "traffic": c["dram_bytes"] if c else None, "traffic_note": note,
            "fit_ms_avg": fit_s * 1e3, "beside": beside}
    return roof


def link_rates(nbytes: int = 1 << 30, reps: int = 3) -> dict:
    """Host<->device copy rates of this machine (pinned host memory, one copy at a time), in GB/s."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dst.copy_(src, non_blocking=True)
            b.record()
            b.synchronize()
            best = min(best, a.elapsed_time(b) * 1e-3)
        out[name] = nbytes / best / 1e9
    del h, d
    return out


def cpu_baseline(frame, seconds_target: float = 15.0, workload: str = "pbpb2m", iterations: int = 0):
    """Time the FP64 oracle with every host core on a bounded sample of the
    frame: the whole frame when a 20k-track probe predicts <= ~2x the target,
    else the first tracks sized for about `seconds_target` seconds.  Returns
    the baseline record and the oracle's fit of the sample (its first tracks)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n = min(20_000, frame.n_tracks)
    sub = frame.subset(0, n)
    t0 = time.perf_counter()
    oracle.fit(sub, oracle.FitConfig(iterations=iterations, **FIT_PARAMS.get(workload, ({}, {}))[1]), threads=cores)
    dt = time.perf_counter() - t0
    predicted = dt * frame.n_clusters / max(sub.n_clusters, 1)
    n2 = frame.n_tracks if predicted <= 2 * seconds_target else int(n * seconds_target / max(dt, 1e-6))
    sub = frame.subset(0, min(n2, frame.n_tracks))
    t0 = time.perf_counter()
    r = oracle.fit(sub, oracle.FitConfig(iterations=iterations, **FIT_PARAMS.get(workload, ({}, {}))[1]), threads=cores)
    dt = time.perf_counter() - t0
    what = "the whole frame" if sub.n_tracks == frame.n_tracks else f"the first {sub.n_tracks} tracks of the frame"
    return {"value": sub.n_clusters / dt, "unit": "clusters/s", "cores": int(r["threads"]), "kind": "oracle",
            "sample": f"{what} ({sub.n_tracks} tracks, {sub.n_clusters} clusters), FP64 C oracle, {dt:.1f} s, "
                      f"one pthread per host core", "tracks_per_s": sub.n_tracks / dt}, r


def parity_block(frame, gpu: dict, orc: dict, workload: str = "pbpb2m", iterations: int = 0) -> dict:
    """The GPU fit of the benchmark frame against the FP64 oracle's fit of the
    same tracks (the cpu_baseline run), element by element with the bars of
    tests/parity.py.  Tracks whose accept flags differ are refitted by the
    oracle with per-cluster chi2, so that flips within the gate window are
    told apart from real mismatches."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    from parity import GATE_WINDOW, TOL_CHI2, TOL_COV, TOL_STATE, compare
    nt = orc["status"].shape[0]
    a, e = int(frame.offsets[0]), int(frame.offsets[nt])
    g = {k: np.asarray(gpu[k][:nt]) for k in ("state", "cov", "chi2", "ndf", "status")}
    g["accept"] = np.asarray(gpu["accept"][a:e])
    off = frame.offsets[:nt + 1] - a
    rep = compare(off, g, orc)
    cfg = oracle.FitConfig(iterations=iterations, **FIT_PARAMS.get(workload, ({}, {}))[1])
    flips = list(rep.accept_mismatch)
    rep.accept_mismatch = []
    gate_excluded = rep.n_gate_excluded
    for t in flips:
        sub = frame.subset(t, t + 1)
        o1 = oracle.fit(sub, cfg, diagnostics=True, threads=1)
        ka, kb = int(off[t]), int(off[t + 1])
        g1 = {k: g[k][t:t + 1] for k in ("state", "cov", "chi2", "ndf", "status")}
        g1["accept"] = g["accept"][ka:kb]
        r1 = compare(sub.offsets, g1, o1)
        gate_excluded += r1.n_gate_excluded
        if r1.accept_mismatch:
            rep.accept_mismatch.append(t)
    st, cnt = np.unique(g["status"], return_counts=True)
    ok = (not rep.status_mismatch and not rep.accept_mismatch and rep.ndf_mismatch == 0
          and rep.max_state < TOL_STATE and rep.max_cov < TOL_COV and rep.max_chi2 < TOL_CHI2)
    return {"oracle": "FP64 C oracle fit of the same tracks in this run", "tracks": int(nt),
            "compared": int(rep.n_compared),
            "gate_excluded": int(gate_excluded), "status_mismatch": len(rep.status_mismatch),
            "accept_mismatch": len(rep.accept_mismatch), "ndf_mismatch": int(rep.ndf_mismatch),
            "max_state_over_sigma": rep.max_state, "max_cov_over_sqrt_diag": rep.max_cov,
            "max_chi2_rel": rep.max_chi2,
            "bars": {"state_over_sigma": TOL_STATE, "cov_over_sqrt_diag": TOL_COV, "chi2_rel": TOL_CHI2,
                     "gate_window_rel": GATE_WINDOW},
            "status_counts": {str(int(s)): int(c) for s, c in zip(st, cnt)}, "ok": bool(ok)}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 oracle on bounded samples of the workload."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n = args.ref_tracks
    if args.workload == "events4096":
        # the first events of the same batch (sizes and tracks are drawn in index order)
        sizes = tpcgen.lognormal_sizes(args.n_events, 800.0, 1.0, 10.0, 20000.0, seed=1000003)
        k = max(1, int(np.searchsorted(np.cumsum(sizes), n, side="right")))
        frame, _ = tpcgen.event_batch(n_events=k, seed=0)
        n = frame.n_tracks
    elif args.workload == "serving":
        frame = tpcgen.generate("detector50k", n_tracks=n, seed=0)  # the first tracks of the frame pool
    else:
        frame = tpcgen.generate(args.workload, n_tracks=n, seed=0)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.fit(frame.subset(0, min(n, 2000)), oracle.FitConfig(**FIT_PARAMS.get(args.workload, ({}, {}))[1]), threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.fit(frame, oracle.FitConfig(**FIT_PARAMS.get(args.workload, ({}, {}))[1]), threads=cores)
    dt = time.perf_counter() - t0
    value = frame.n_clusters * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "clusters/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                   "sample": f"first {n} tracks ({frame.n_clusters} clusters) of the workload per step"},
        "cpu_baseline": {"value": value, "unit": "clusters/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {n} tracks ({frame.n_clusters} clusters) per step"},
        "e2e": {"value": value, "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def gpu_index(local: int) -> int:
    v = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    return int(v) if v.isdigit() else local


def reduce_max(dist, torch, x: float) -> float:
    """Max over the ranks (timing only; the data path has no collective)."""
    from paper_2402_01205_gb300 import replicas
    return replicas.max_over_ranks(x, device="cuda") if dist else x


def reduce_sum(dist, torch, x: float) -> float:
    from paper_2402_01205_gb300 import replicas
    return replicas.sum_over_ranks(x, device="cuda") if dist else x


def frame_seed(rank: int, ws: int) -> int:
    """The seed of the frame this rank fits: one independent time frame per
    rank, frames dealt round robin over the ranks (the paper's distribution of
    time frames over GPUs without GPU intercommunication, Sec. 6)."""
    from paper_2402_01205_gb300 import replicas
    mine = replicas.shard_round_robin(ws, rank, ws)
    return mine[0]


def run_events(args, ws, rank, local, T, torch, dist, probe, leg: bool = False):
    """Batched uneven events: the autotuned batch graph vs one launch per event.
    As a leg of the default run (``leg``): fewer steps, no end-to-end or CPU
    arm, and a compact record returned instead of a printed line."""
    from paper_2402_01205_gb300 import autotune
    frame, ev = tpcgen.event_batch(n_events=args.n_events, seed=frame_seed(rank, ws))
    nt, nc = frame.n_tracks, frame.n_clusters
    names = ("offsets", "x", "y", "z", "sy2", "sz2", "row")

    class F:
        pass

    dev = F()
    for k in names:
        setattr(dev, k, torch.from_numpy(np.ascontiguousarray(getattr(frame, k))).cuda())
    props = torch.cuda.get_device_properties(local)
    table = autotune.load(args.tune_table) if args.tune_table else {}
    entry = autotune.lookup(table, props.name, props.multi_processor_count, nt)
    tuned_now = entry is None
    if tuned_now:
        entry = autotune.tune(T, dev, reps=1 if leg else 3, device=local)
        if args.tune_table and rank == 0:
            autotune.save(args.tune_table, autotune.table_key(props.name, props.multi_processor_count, nt), entry)
    cfg = autotune.config_for(entry)
    fx = T.Fitter(device=local, **cfg)
    stream = torch.cuda.Stream()
    # batched arm: one captured launch sequence over all events per step
    batch = T.Batch(fx, dev)
    for _ in range(args.warmup):
        batch.launch(stream)
    batch.sync()
    clocks = ClockSampler(gpu_index(local))
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        batch.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    batch.sync()
    ms = reduce_max(dist, torch, e0.elapsed_time(e1))
    nc_all = reduce_sum(dist, torch, float(nc))
    nt_all = reduce_sum(dist, torch, float(nt))
    value = nc_all * args.steps / (ms * 1e-3)
    res_b = {k: v.clone() for k, v in batch.res.items()}
    # kernel split of the same launch sequence (event-timed plain fit of the whole batch frame)
    res_t = T.alloc_result(nt, nc, device=torch.device("cuda", local))
    fx.reset_timing()
    for _ in range(3):
        fx.fit_async(dev, res_t, stream=stream)
    fx.sync()
    tm = fx.timing()
    # per-event arm: one plain launch sequence per event, in event order, on one stream
    res_e = T.alloc_result(nt, nc, device=torch.device("cuda", local))
    views = T.EventViews(dev, res_e, ev)
    views.fit_async(fx, stream)
    fx.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0 = time.perf_counter()
    p0.record(stream)
    for _ in range(args.per_event_steps):
        views.fit_async(fx, stream)
    p1.record(stream)
    torch.cuda.synchronize()
    host_s = time.perf_counter() - h0
    ms_pe = reduce_max(dist, torch, p0.elapsed_time(p1))
    same = all(torch.equal(res_b[k], res_e[k]) or (k in ("state", "cov") and torch.equal(
        torch.nan_to_num(res_b[k], nan=7.0), torch.nan_to_num(res_e[k], nan=7.0))) for k in res_b)
    status = res_b["status"].cpu().numpy()
    ok = status == 0
    lens = np.diff(frame.offsets)
    nc_fit = int(lens[ok].sum())
    seq_s = tm["total_ms_sum"] / max(tm["n_timed"], 1) * 1e-3
    fit_s = tm["fit_ms_sum"] / max(tm["n_timed"], 1) * 1e-3
    roofline = fit_roofline(nc, nt, nc_fit, fit_s, (tm["fit_grid"], tm["fit_block"]), probe,
                            props.multi_processor_count, clk.get("sm_mhz"))
    if leg:
        sizes = np.diff(ev)
        out = {"workload": "events4096", "description": WORKLOADS["events4096"], "n_events": len(sizes),
               "n_tracks": nt, "n_clusters": nc, "tracks_per_event_median": float(np.median(sizes)),
               "batch": {"clusters_per_s": value, "tracks_per_s": nt_all * args.steps / (ms * 1e-3),
                         "ms_per_step": ms / args.steps, "steps": args.steps,
                         "launch": "tpcfit_batch graph replay (one captured launch sequence per step)"},
               "per_event": {"clusters_per_s": nc_all * args.per_event_steps / (ms_pe * 1e-3),
                             "ms_per_step": ms_pe / args.per_event_steps, "steps": args.per_event_steps,
                             "launch": "tpcfit_fit_async per event, one stream"},
               "speedup_of_batch": (ms_pe / args.per_event_steps) / (ms / args.steps),
               "results_identical_to_batch": bool(same), "autotuned": cfg, "autotune_ms": entry["ms"],
               "autotune_candidates": entry.get("all"), "fit_roofline_frac": roofline["frac"], "clocks": clk}
        batch.close()
        fx.close()
        return out
    e2e = None
    if args.e2e_steps > 0:
        host = F()
        for k in names:
            t = torch.empty(getattr(dev, k).shape, dtype=getattr(dev, k).dtype, pin_memory=True)
            t.copy_(torch.from_numpy(np.ascontiguousarray(getattr(frame, k))))
            setattr(host, k, t)
        hres = T.alloc_result(nt, nc, pinned=True)
        for _ in range(max(3, args.warmup)):  # untimed warm-up calls
            fx.fit(host, hres)
        if dist:
            dist.barrier()
        with host_timed():
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                fx.fit(host, hres)
                _ = float(hres["chi2"][0])
            dt = time.perf_counter() - t0
        dt = reduce_max(dist, torch, dt)
        e2e = {"value": nc_all * args.e2e_steps / dt, "unit": "clusters/s",
               "h2d_bytes_per_step": int(21 * nc + 8 * (nt + 1)), "d2h_bytes_per_step": int(100 * nt + nc),
               "ms_per_step": dt / args.e2e_steps * 1e3,
               "path": "tpcfit_fit of the concatenated events, TPCFIT_MEM_HOST pinned, chunked overlap"}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, _ = cpu_baseline(frame, workload=args.workload)
    if rank == 0:
        sizes = np.diff(ev)
        line = {
            "metric": "clusters/s fitted on 1 GB300, batched uneven events (FP32 fit, FP64 innovation inverse "
                      "and chi2)",
            "value": value, "unit": "clusters/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "events4096", "description": WORKLOADS["events4096"], "n_events": len(sizes),
                       "n_tracks": nt, "n_clusters": nc, "tracks_per_event_median": float(np.median(sizes)),
                       "tracks_per_event_min": int(sizes.min()), "tracks_per_event_max": int(sizes.max()),
                       "tracks_fitted_ok": int(ok.sum()), "l2": f"inputs {21 * nc / 1e9:.1f} GB > L2; no flush",
                       "parallelism": f"replicas x{ws}", "launch": "tpcfit_batch graph replay",
                       "autotuned": cfg, "autotune_ms": entry["ms"], "tuned_in_this_run": tuned_now,
                       "autotune_candidates": entry.get("all")},
            "tracks_per_s": nt_all * args.steps / (ms * 1e-3),
            "per_event": {"value": nc_all * args.per_event_steps / (ms_pe * 1e-3), "unit": "clusters/s",
                          "ms_per_step": ms_pe / args.per_event_steps, "steps": args.per_event_steps,
                          "host_ms_per_step": host_s / args.per_event_steps * 1e3,
                          "launch": "tpcfit_fit_async per event (memset + 4 kernels + 1 copy each), one stream",
                          "speedup_of_batch": (ms_pe / args.per_event_steps) / (ms / args.steps),
                          "results_identical_to_batch": bool(same)},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(tm["kernel_launches"]) * args.steps,
            "clocks": clk,
            "kernel_ms": {"prepare": tm["prepare_ms_sum"] / tm["n_timed"], "sort": tm["sort_ms_sum"] / tm["n_timed"],
                          "fit": tm["fit_ms_sum"] / tm["n_timed"], "sequence": seq_s * 1e3},
        }
        print(json.dumps(line), flush=True)
    batch.close()
    fx.close()
    if dist:
        dist.destroy_process_group()
    return 0


SERVE_MEDIAN, SERVE_SIGMA, SERVE_LO, SERVE_HI = 20e6, 0.6, 1e6, 120e6


def serving_pool(rank: int, n_frames: int, pool_tracks: int = 1_100_000, seed: int = 0):
    """One pre-generated frame and n_frames windows of it whose cluster counts
    follow the serving size law.  Returns (frame, [(t0, t1), ...])."""
    big = tpcgen.generate("detector50k", n_tracks=pool_tracks, seed=rank)
    want = tpcgen.lognormal_sizes(n_frames, SERVE_MEDIAN, SERVE_SIGMA, SERVE_LO, SERVE_HI, seed=seed + 77)
    rng = np.random.default_rng(seed + 78)
    off = big.offsets
    wins = []
    for c in want:
        c = min(int(c), int(off[-1]) - 1)
        # last start whose window of c clusters still fits
        last = int(np.searchsorted(off, off[-1] - c, side="right")) - 1
        t0 = int(rng.integers(0, max(last, 0) + 1))
        t1 = int(np.searchsorted(off, off[t0] + c, side="left"))
        wins.append((t0, max(t1, t0 + 1)))
    return big, wins


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else None


def run_serving(args, ws, rank, local, T, torch, dist, probe, leg: bool = False):
    """Served frames (tpcfit_submit/poll) vs sequential plain fits (tpcfit_fit).
    As a leg of the default run (``leg``): the Poisson window only (served,
    then the same schedule as sequential plain fits), a compact record
    returned instead of a printed line."""
    big, wins = serving_pool(rank, args.serve_pool)
    names = ("offsets", "x", "y", "z", "sy2", "sz2", "row")

    class F:
        pass

    pinned = {}
    for k in names[1:]:
        a = getattr(big, k)
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:1]).dtype, pin_memory=True)
        t.copy_(torch.from_numpy(a))
        pinned[k] = t
    frames = []
    for t0, t1 in wins:
        c0, c1 = int(big.offsets[t0]), int(big.offsets[t1])
        f = F()
        o = torch.empty(t1 - t0 + 1, dtype=torch.int64, pin_memory=True)
        o.copy_(torch.from_numpy(big.offsets[t0:t1 + 1] - c0))
        f.offsets = o
        for k in names[1:]:
            setattr(f, k, pinned[k][c0:c1])
        f.n_tracks, f.n_clusters = t1 - t0, c1 - c0
        frames.append(f)
    max_nt = max(f.n_tracks for f in frames)
    max_nc = max(f.n_clusters for f in frames)
    ring = [T.alloc_result(max_nt, max_nc, pinned=True) for _ in range(16)]

    def res_for(slot, f):
        return {k: (v[:f.n_clusters] if k == "accept" else v[:f.n_tracks]) for k, v in ring[slot].items()}

    n_req = max(1, int(round(args.serve_seconds * args.serve_rate)))
    arrivals = tpcgen.poisson_arrivals(n_req, args.serve_rate, seed=rank + 79)
    pick = np.random.default_rng(rank + 80).integers(0, len(frames), size=n_req)
    budget = 120 << 30

    def served(arr):
        lat, t_done = [None] * len(arr), [0.0] * len(arr)
        with T.Fitter(device=local, hbm_budget_bytes=budget, max_slots=8) as fx:
            fx.wait(fx.submit(frames[0], res_for(0, frames[0])))  # warm-up: pool, streams, kernels
            out = {}
            with host_timed():
                t0 = T.now() + 0.05
                for i, a in enumerate(arr):
                    slot = i % len(ring)
                    if slot in out:
                        tk, j = out.pop(slot)
                        st, td = fx.wait(tk)
                        assert st == T.DONE, st
                        lat[j], t_done[j] = td - (t0 + arr[j]), td
                    d = t0 + a - T.now()
                    if d > 0:
                        time.sleep(d)
                    f = frames[pick[i]]
                    out[slot] = (fx.submit(f, res_for(slot, f)), i)
                for tk, j in out.values():
                    st, td = fx.wait(tk)
                    assert st == T.DONE, st
                    lat[j], t_done[j] = td - (t0 + arr[j]), td
            eng = fx.serve_stats()
        eng["parts_per_launch_mean"] = eng["parts"] / max(eng["launches"], 1)
        return lat, max(t_done) - (t0 + arr[0]), eng

    def sequential(arr):
        lat, t_end = [None] * len(arr), 0.0
        with T.Fitter(device=local) as fx, host_timed():
            fx.fit(frames[0], res_for(0, frames[0]))
            t0 = T.now() + 0.05
            for i, a in enumerate(arr):
                d = t0 + a - T.now()
                if d > 0:
                    time.sleep(d)
                f = frames[pick[i]]
                fx.fit(f, res_for(i % len(ring), f))
                t_end = T.now()
                lat[i] = t_end - (t0 + a)
        return lat, t_end - (t0 + arr[0])

    def unloaded(f, reps=3):
        """Latency of one frame with nothing else in flight: served, and plain fit."""
        out = {}
        with T.Fitter(device=local, hbm_budget_bytes=budget, max_slots=8) as fx:
            fx.wait(fx.submit(f, res_for(0, f)))
            ts = []
            for _ in range(reps):
                t0 = T.now()
                ts.append(fx.wait(fx.submit(f, res_for(0, f)))[1] - t0)
            out["served_ms"] = 1e3 * min(ts)
        with T.Fitter(device=local) as fx:
            fx.fit(f, res_for(0, f))
            ts = []
            for _ in range(reps):
                t0 = T.now()
                fx.fit(f, res_for(0, f))
                ts.append(T.now() - t0)
            out["plain_fit_ms"] = 1e3 * min(ts)
        out["n_clusters"] = f.n_clusters
        out["h2d_floor_ms"] = 1e3 * (21 * f.n_clusters + 8 * f.n_tracks) / 211e9
        return out

    ncl = np.array([frames[k].n_clusters for k in pick], dtype=np.float64)
    ntr = np.array([frames[k].n_tracks for k in pick], dtype=np.float64)

    def summary(lat, span, cl, tr):
        ms = [x * 1e3 for x in lat]
        return {"p50_ms": percentile(ms, 50), "p90_ms": percentile(ms, 90), "p99_ms": percentile(ms, 99),
                "p999_ms": percentile(ms, 99.9), "max_ms": max(ms),
                "mean_ms": float(np.mean(ms)), "clusters_per_s": cl / span, "tracks_per_s": tr / span,
                "frames": len(lat), "span_s": span}

    if leg:
        clocks = ClockSampler(gpu_index(local))
        clocks.start()
        lat_s, span_s, eng = served(arrivals)
        clk = clocks.stop()
        lat_q, span_q = sequential(arrivals)
        return {"workload": "serving", "description": WORKLOADS["serving"], "rate_hz": args.serve_rate,
                "seconds": args.serve_seconds, "frames_submitted": n_req, "pool_frames": len(frames),
                "clusters_per_frame_median": float(np.median(ncl)), "clusters_per_frame_max": float(ncl.max()),
                "hbm_budget_bytes": budget, "max_slots": 8,
                "latency": "arrival on the seeded schedule to results in pinned host memory",
                "served": dict(summary(lat_s, span_s, ncl.sum(), ntr.sum()), engine=eng),
                "sequential_plain_fit": summary(lat_q, span_q, ncl.sum(), ntr.sum()), "clocks": clk}
    by_size = sorted(range(len(frames)), key=lambda k: frames[k].n_clusters)
    unloaded_lat = {"largest": unloaded(frames[by_size[-1]]), "median": unloaded(frames[by_size[len(by_size) // 2]])}
    if dist:
        dist.barrier()
    clocks = ClockSampler(gpu_index(local))
    clocks.start()
    lat_s, span_s, eng = served(arrivals)
    clk = clocks.stop()
    lat_q, span_q = sequential(arrivals)
    # capacity: every frame of the schedule due at once
    n_cap = min(n_req, 4 * len(frames))
    zero = np.zeros(n_cap)
    lat_cs, span_cs, eng_cap = served(zero)
    lat_cq, span_cq = sequential(zero)
    cap_cl = float(ncl[:n_cap].sum())
    # device-only fit time of each pool frame, resident in HBM
    dev_ms, fit_ms, fit_cl, fit_tr = [], 0.0, 0, 0
    with T.Fitter(device=local) as fx:
        for f in frames:
            g = F()
            for k in names:
                setattr(g, k, getattr(f, k).cuda())
            r = T.alloc_result(f.n_tracks, f.n_clusters, device=torch.device("cuda", local))
            fx.fit_async(g, r)
            fx.sync()
            tm = fx.timing()
            dev_ms.append(tm["total_ms"])
            ok = (r["status"] == 0).cpu().numpy()
            lens = np.diff(f.offsets.numpy())
            fit_ms += tm["fit_ms"]
            fit_cl += int(lens[ok].sum())
            fit_tr += f.n_tracks
            del g, r
    nc_pool = sum(f.n_clusters for f in frames)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roofline = fit_roofline(nc_pool, fit_tr, fit_cl, fit_ms * 1e-3, (tm["fit_grid"], tm["fit_block"]), probe, sms,
                            clk.get("sm_mhz"))
    roofline["over"] = f"one device-resident fit of each of the {len(frames)} pool frames"
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, _ = cpu_baseline(big)
    sustained = float(ncl.sum()) / span_s
    value = reduce_sum(dist, torch, sustained)

    if rank == 0:
        line = {
            "metric": "sustained clusters/s and p50/p99 frame latency (arrival to results in caller memory) of "
                      "served time frames on 1 GB300",
            "value": value, "unit": "clusters/s", "n_gpus": ws, "steps": n_req, "warmup": 1,
            "ms_per_step": span_s / n_req * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "serving", "description": WORKLOADS["serving"], "rate_hz": args.serve_rate,
                       "seconds": args.serve_seconds, "frames_submitted": n_req, "pool_frames": len(frames),
                       "clusters_per_frame_median": float(np.median(ncl)), "clusters_per_frame_max": float(ncl.max()),
                       "hbm_budget_bytes": budget, "max_slots": 8, "result_ring": len(ring),
                       "l2": "frames of 1-120 M clusters, copied in per request; no flush",
                       "parallelism": f"replicas x{ws}"},
            "latency": {"served": dict(summary(lat_s, span_s, ncl.sum(), ntr.sum()), engine=eng),
                        "sequential_plain_fit": summary(lat_q, span_q, ncl.sum(), ntr.sum())},
            "capacity": {"frames": n_cap,
                         "served": dict(summary(lat_cs, span_cs, cap_cl, float(ntr[:n_cap].sum())), engine=eng_cap),
                         "sequential_plain_fit": summary(lat_cq, span_cq, cap_cl, float(ntr[:n_cap].sum()))},
            "unloaded_latency": unloaded_lat,
            "device_only_fit_ms": {"p50": percentile(dev_ms, 50), "p99": percentile(dev_ms, 99),
                                   "note": "one pool frame resident in HBM, launch sequence time"},
            "e2e": {"value": sustained, "unit": "clusters/s", "h2d_bytes_per_step": int(21 * ncl.mean() + 8 * ntr.mean()),
                    "d2h_bytes_per_step": int(100 * ntr.mean() + ncl.mean()),
                    "path": "tpcfit_submit / tpcfit_wait, pinned host frames and results"},
            "roofline": roofline, "cpu_baseline": cpu,
            "gpu_launches": 4 * n_req,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def tracking_inputs(n_tracks: int, rank: int, seed: int = 0):
    f = tpcgen.generate("detector50k", n_tracks=n_tracks, seed=rank, truth=True)
    first = f.offsets[:-1]
    seed_cov = np.array([0.01, 0.01, 1e-4, 1e-4, 0.01])
    st = (f.truth[first] + np.random.default_rng(seed + 91).normal(0, 1, (f.n_tracks, 5)) * np.sqrt(seed_cov) * 0.3)
    sec = np.repeat(f.sector, np.diff(f.offsets)).astype(np.uint8)
    return f, st.astype(np.float32), sec


def run_tracking(args, ws, rank, local, T, torch, dist, probe):
    """Track following + gather + fit (the tracking chain) on the GPU."""
    import types
    n_tracks = args.n_tracks or 50_000
    f, st, sec = tracking_inputs(n_tracks, rank)
    nc, nt = f.n_clusters, f.n_tracks
    first = f.offsets[:-1]
    dev = types.SimpleNamespace(**{k: torch.from_numpy(np.ascontiguousarray(getattr(f, k))).cuda()
                                   for k in ("x", "y", "z", "sy2", "sz2", "row")}, sectors=torch.from_numpy(sec).cuda())
    seeds = dict(state=torch.from_numpy(st).cuda(), row=torch.from_numpy(np.ascontiguousarray(f.row[first])).cuda(),
                 sector=torch.from_numpy(np.ascontiguousarray(f.sector)).cuda())
    fx = T.Fitter(device=local)
    stream = torch.cuda.Stream()

    def chain():
        tr = fx.follow(dev, seeds, stream=stream)
        fr = fx.gather_tracks(dev, tr, stream=stream)  # blocks on `stream`
        fx.fit_async(fr, T.alloc_result(fr.offsets.numel() - 1, fr.x.numel(), device=torch.device("cuda", local)),
                     stream=stream)
        return tr

    for _ in range(args.warmup):
        tr = chain()
    fx.sync()
    torch.cuda.synchronize()
    # following alone
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        tr = fx.follow(dev, seeds, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_follow = reduce_max(dist, torch, e0.elapsed_time(e1)) / args.steps
    # the whole chain
    clocks = ClockSampler(gpu_index(local))
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(args.steps):
        tr = chain()
    fx.sync()
    c1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = reduce_max(dist, torch, c0.elapsed_time(c1)) / args.steps
    nc_all = reduce_sum(dist, torch, float(nc))
    # efficiency and purity against the generator's truth
    att = tr["att"].cpu().numpy()
    own = wrong = 0
    for t in range(0, nt, max(1, nt // 20000)):
        a = att[t][att[t] >= 0]
        ok = (a >= f.offsets[t]) & (a < f.offsets[t + 1])
        own += int(ok.sum())
        wrong += int((~ok).sum())
    sample_true = int(sum(f.offsets[t + 1] - f.offsets[t] for t in range(0, nt, max(1, nt // 20000))))
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        k = min(nt, 20_000)
        hits = types.SimpleNamespace(y=f.y, z=f.z, sy2=f.sy2, sz2=f.sz2, row=f.row, sectors=sec)
        sd = dict(state=st[:k].astype(np.float64), row=f.row[first[:k]], sector=f.sector[:k])
        t0 = time.perf_counter()
        oracle.follow(hits, sd, oracle.FitConfig(), oracle.FollowConfig())
        dt = time.perf_counter() - t0
        cl = float(f.offsets[k])
        cpu = {"value": cl / dt, "unit": "clusters/s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"FP64 follower on the first {k} seeds ({int(cl)} clusters of their tracks) with the "
                         f"whole frame's clusters bucketed, {dt:.1f} s (includes the bucketing)"}
    peaks, peak_src = measured_peaks()
    follow_bytes = 16 * nc + 24 * nt  # cell build reads y, z, sy2, sz2 (16 B/cluster); seeds + results per track
    if rank == 0:
        line = {
            "metric": "clusters/s tracked on 1 GB300 (track following + gather + fit, FP32 with FP64 gate)",
            "value": nc_all / (ms * 1e-3), "unit": "clusters/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "tracking", "description": WORKLOADS["tracking"], "n_tracks": nt, "n_clusters": nc,
                       "parallelism": f"replicas x{ws}", "l2": f"inputs {21 * nc / 1e9:.2f} GB; no flush"},
            "tracks_per_s": reduce_sum(dist, torch, float(nt)) / (ms * 1e-3),
            "follow_only": {"ms": ms_follow, "clusters_per_s": nc / (ms_follow * 1e-3),
                            "hbm_frac_of_min_bytes": follow_bytes / (ms_follow * 1e-3) / 1e9 / peaks["hbm_gbs"]},
            "efficiency": own / max(sample_true, 1), "purity": own / max(own + wrong, 1),
            "roofline": {"bound": "alu", "kernel": "k_follow + k_fit", "unit": "GB/s (minimum bytes)",
                         "achieved": follow_bytes / (ms_follow * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                         "frac": follow_bytes / (ms_follow * 1e-3) / 1e9 / peaks["hbm_gbs"], "traffic": None,
                         "traffic_note": "no ncu capture of k_follow; latency-bound like the fit (one thread per track)",
                         "peak_source": peak_src},
            "cpu_baseline": cpu,
            "e2e": None,
            "gpu_launches": 16 * args.steps,  # follow 6 (cells 5 + k_follow), gather 6, fit 4
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    fx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pbpb2m", choices=sorted(WORKLOADS))
    ap.add_argument("--n-tracks", type=int, default=None, help="override the workload's track count (testing)")
    ap.add_argument("--e2e-steps", type=int, default=20, help="timed end-to-end steps (the mean over them is reported)")
    ap.add_argument("--ref-tracks", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rans-steps", type=int, default=5, help="pbpb2m: timed rANS encode/decode calls per stream")
    ap.add_argument("--block-threads", type=int, default=0, help="pbpb2m: fit kernel block size (0 = library default)")
    ap.add_argument("--blocks-per-sm", type=int, default=0, help="pbpb2m: resident fit blocks per SM (0 = default)")
    ap.add_argument("--fit-iterations", type=int, default=0, help="pbpb2m(_eloss): seed iterations of the fit (variant)")
    ap.add_argument("--n-events", type=int, default=4096, help="events4096: number of events (testing)")
    ap.add_argument("--per-event-steps", type=int, default=3, help="events4096: timed steps of the per-event arm")
    ap.add_argument("--tune-table", default=None, help="events4096: JSON tune table to read / extend")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serving: length of the arrival schedule")
    ap.add_argument("--serve-rate", type=float, default=50.0, help="serving: frames/s")
    ap.add_argument("--serve-pool", type=int, default=64, help="serving: distinct frames in the replayed pool")
    ap.add_argument("--no-legs", action="store_true",
                    help="pbpb2m: leave out the batched-events and serving legs of the default line")
    ap.add_argument("--leg-serve-seconds", type=float, default=10.0, help="serving leg: length of the arrival schedule")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import paper_2402_01205_gb300 as T
    from paper_2402_01205_gb300 import _build
    _build.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    probe = T.probe_fma_rates(local)
    if args.workload == "events4096":
        return run_events(args, ws, rank, local, T, torch, dist, probe)
    if args.workload == "serving":
        return run_serving(args, ws, rank, local, T, torch, dist, probe)
    if args.workload == "tracking":
        return run_tracking(args, ws, rank, local, T, torch, dist, probe)
    kw = {} if args.n_tracks is None else {"n_tracks": args.n_tracks}
    frame = tpcgen.generate(args.workload, seed=frame_seed(rank, ws), **kw)
    nt, nc = frame.n_tracks, frame.n_clusters
    names = ("offsets", "x", "y", "z", "sy2", "sz2", "row")

    class F:
        pass

    dev = F()
    for k in names:
        setattr(dev, k, torch.from_numpy(np.ascontiguousarray(getattr(frame, k))).cuda())
    fx = T.Fitter(device=local, block_threads=args.block_threads, blocks_per_sm=args.blocks_per_sm,
                  fit_iterations=args.fit_iterations, **FIT_PARAMS.get(args.workload, ({}, {}))[0])
    res = T.alloc_result(nt, nc, device=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    for _ in range(args.warmup):
        fx.fit_async(dev, res, stream=stream)
    fx.sync()
    fx.reset_timing()
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        fx.fit_async(dev, res, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    tm = fx.timing()
    ms = reduce_max(dist, torch, ms)
    nc_all = reduce_sum(dist, torch, float(nc))
    value = nc_all * args.steps / (ms * 1e-3)
    status = res["status"].cpu().numpy()
    ok = status == 0
    lens = np.diff(frame.offsets)
    nc_fit = int(lens[ok].sum())
    fit_s = tm["fit_ms_sum"] / max(tm["n_timed"], 1) * 1e-3
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    variant = ("eloss" if args.workload == "pbpb2m_eloss" else "") + (f"iter{args.fit_iterations}" if args.fit_iterations
                                                                       else "")
    roofline = fit_roofline(nc, nt, nc_fit, fit_s, (tm["fit_grid"], tm["fit_block"]), probe, sms, clk.get("sm_mhz"),
                            variant, passes=1 + args.fit_iterations)
    roofline["fp32_fma_peak_per_s"] = probe["fp32_fma_per_s"]
    # the same steps with the track-model compression residual codes written (4 B per cluster more)
    res_r = T.alloc_result(nt, nc, device=torch.device("cuda", local), residuals=True)
    for _ in range(2):
        fx.fit_async(dev, res_r, stream=stream)
    fx.sync()
    fx.reset_timing()
    n_res = max(3, min(args.steps, 20))
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(n_res):
        fx.fit_async(dev, res_r, stream=stream)
    r1.record(stream)
    torch.cuda.synchronize()
    ms_res = reduce_max(dist, torch, r0.elapsed_time(r1))
    tm_res = fx.timing()
    with_residuals = {"value": nc_all * n_res / (ms_res * 1e-3), "unit": "clusters/s", "steps": n_res,
                      "ms_per_step": ms_res / n_res, "fit_ms": tm_res["fit_ms_sum"] / max(tm_res["n_timed"], 1),
                      "extra_bytes_per_cluster": 4,
                      "what": "int16 residual codes of every cluster against the fitted helix (y and z)"}
    # rANS entropy coding of the residual codes (both streams), blocking calls timed whole
    codec = None
    if args.rans_steps > 0:
        peaks, _ = measured_peaks()
        enc_s, dec_s, sizes = [], [], []
        outs = {}
        for k in ("res_y", "res_z"):
            outs[k] = fx.rans_encode(res_r[k], stream=stream)
            fx.rans_decode(outs[k][0], outs[k][1], nc, stream=stream)
        dec = torch.empty(nc, dtype=torch.int16, device=torch.device("cuda", local))
        for _ in range(args.rans_steps):
            for k in ("res_y", "res_z"):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                o, sz = fx.rans_encode(res_r[k], out=outs[k][0], stream=stream)
                enc_s.append(time.perf_counter() - t0)
                t0 = time.perf_counter()
                fx.rans_decode(o, sz, nc, out=dec, stream=stream)
                dec_s.append(time.perf_counter() - t0)
                sizes.append(sz)
        ok_rt = bool(torch.equal(dec, res_r["res_z"]))
        e_ms, d_ms = 1e3 * statistics.median(enc_s), 1e3 * statistics.median(dec_s)
        mean_size = float(np.mean(sizes))
        dec_bytes = mean_size + 2 * nc  # container read + codes written
        codec = {"encode_gcodes_s": nc / (e_ms * 1e-3) / 1e9, "decode_gcodes_s": nc / (d_ms * 1e-3) / 1e9,
                 "encode_ms": e_ms, "decode_ms": d_ms, "codes_per_stream": nc, "streams": 2,
                 "bits_per_code": 8 * mean_size / nc, "raw_bits_per_code": 16,
                 "decode_hbm": {"achieved_gbs": dec_bytes / (d_ms * 1e-3) / 1e9, "peak_gbs": peaks["hbm_gbs"],
                                "frac": dec_bytes / (d_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                                "bytes": "container read + 2 B per code written"},
                 "round_trip_identical": ok_rt, "calls": "tpcfit_rans_encode / tpcfit_rans_decode, blocking, "
                 "median of %d calls per stream" % args.rans_steps}
        del outs, dec
    del res_r
    # the two-filter smoother variant (per-cluster smoothed states, 80 B per cluster written)
    smoother = None
    if args.workload == "pbpb2m" and args.fit_iterations == 0:
        res_s = T.alloc_result(nt, nc, device=torch.device("cuda", local), smoothed=True)
        fx.fit_async(dev, res_s, stream=stream)
        fx.sync()
        fx.reset_timing()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_sm = 3
        s0.record(stream)
        for _ in range(n_sm):
            fx.fit_async(dev, res_s, stream=stream)
        s1.record(stream)
        torch.cuda.synchronize()
        ms_sm = reduce_max(dist, torch, s0.elapsed_time(s1))
        tm_s = fx.timing()
        smoother = {"value": nc_all * n_sm / (ms_sm * 1e-3), "unit": "clusters/s", "steps": n_sm,
                    "ms_per_step": ms_sm / n_sm, "kernel_ms": tm_s["fit_ms_sum"] / max(tm_s["n_timed"], 1),
                    "what": "two-filter smoother: forward predictions stored, backward filter, 5x5 combination at "
                            "every cluster; smoothed state and covariance written per cluster (80 B)"}
        del res_s
    # end to end through the C-ABI: pinned host frame in, pinned host results out
    e2e = None
    if args.e2e_steps > 0:
        host = F()
        for k in names:
            t = torch.empty(getattr(dev, k).shape, dtype=getattr(dev, k).dtype, pin_memory=True)
            t.copy_(torch.from_numpy(np.ascontiguousarray(getattr(frame, k))))
            setattr(host, k, t)
        hres = T.alloc_result(nt, nc, pinned=True)
        for _ in range(max(3, args.warmup)):  # untimed warm-up calls: staging buffers, pinned pages
            fx.fit(host, hres)
        if dist:
            dist.barrier()
        step_ms = []
        with host_timed():
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                ts = time.perf_counter()
                fx.fit(host, hres)
                _ = float(hres["chi2"][0])  # the step's result read on the host
                step_ms.append(round(1e3 * (time.perf_counter() - ts), 3))
            dt = time.perf_counter() - t0
        dt = reduce_max(dist, torch, dt)
        h2d_b, d2h_b = int(21 * nc + 8 * (nt + 1)), int(100 * nt + nc)
        # the same frame without x: its clusters lie on the pad-row planes, and
        # the library derives x from the rows on the device (17 B per cluster copied)
        ref_state, ref_accept = hres["state"].clone(), hres["accept"].clone()
        nox = F()
        for k in names:
            setattr(nox, k, None if k == "x" else getattr(host, k))
        for _ in range(max(3, args.warmup)):
            fx.fit(nox, hres)
        nox_ms = []
        with host_timed():
            for _ in range(args.e2e_steps):
                ts = time.perf_counter()
                fx.fit(nox, hres)
                _ = float(hres["chi2"][0])
                nox_ms.append(round(1e3 * (time.perf_counter() - ts), 3))
        nox_s = reduce_max(dist, torch, sum(nox_ms) * 1e-3)
        nox_same = bool(torch.equal(ref_state.view(torch.int32), hres["state"].view(torch.int32))  # bitwise (NaN too)
                        and torch.equal(ref_accept, hres["accept"]))
        del ref_state, ref_accept
        link = link_rates()
        e2e = {"value": nc_all * args.e2e_steps / dt, "unit": "clusters/s",
               "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b,
               "ms_per_step": dt / args.e2e_steps * 1e3, "step_ms": step_ms,
               "median_ms": float(np.median(step_ms)),
               "path": "tpcfit_fit, TPCFIT_MEM_HOST pinned, chunked overlap",
               "link": dict(link, floor_ms=1e3 * h2d_b / (link["h2d_gbs"] * 1e9),
                            note="pinned copies of 1 GiB timed on this box; floor = the frame's host-to-device "
                                 "bytes at that rate")}
        e2e["without_x"] = {
            "value": nc_all * args.e2e_steps / nox_s, "unit": "clusters/s", "median_ms": float(np.median(nox_ms)),
            "step_ms": nox_ms, "h2d_bytes_per_step": int(17 * nc + 8 * (nt + 1)), "d2h_bytes_per_step": d2h_b,
            "what": "the same frame passed without x (its clusters lie on the pad-row planes: x derived on the device "
                    "from the rows)", "results_identical_to_e2e": nox_same}
    cpu, parity = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        gpu_host = {k: res[k].cpu().numpy() for k in ("state", "cov", "chi2", "ndf", "status", "accept")}
        cpu, orc = cpu_baseline(frame, workload=args.workload, iterations=args.fit_iterations)
        parity = parity_block(frame, gpu_host, orc, args.workload, args.fit_iterations)
        del gpu_host, orc
    # the other two workloads of the metric, shortened, on this GPU after the timed steps
    legs = {}
    if ws == 1 and not args.no_legs and args.workload == "pbpb2m":
        import copy
        la = copy.copy(args)
        la.steps, la.warmup, la.per_event_steps, la.e2e_steps, la.n_events = 5, 2, 1, 0, 4096
        la.serve_seconds, la.tune_table = args.leg_serve_seconds, None
        legs["events4096"] = run_events(la, ws, rank, local, T, torch, None, probe, leg=True)
        legs["serving"] = run_serving(la, ws, rank, local, T, torch, None, probe, leg=True)
    if rank == 0:
        srv = legs.get("serving", {}).get("served", {})
        line = {
            "metric": METRIC,
            "value": value, "unit": "clusters/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "n_tracks": nt,
                       "fit_iterations": args.fit_iterations,
                       "n_clusters": nc, "tracks_fitted_ok": int(ok.sum()), "l2": "inputs 4.2 GB > L2; no flush",
                       "parallelism": f"replicas x{ws}", "fit_grid": tm["fit_grid"], "fit_block": tm["fit_block"],
                       "fit_regs": tm["fit_regs"]},
            "tracks_per_s": nt * ws * args.steps / (ms * 1e-3),
            "metrics": {"clusters_per_s": value, "tracks_per_s": nt * ws * args.steps / (ms * 1e-3),
                        "oracle_error": None if parity is None else {
                            k: parity[k] for k in ("max_state_over_sigma", "max_cov_over_sqrt_diag", "max_chi2_rel",
                                                   "ok")},
                        "p50_ms": srv.get("p50_ms"), "p99_ms": srv.get("p99_ms"),
                        "latency_from": "the serving leg (Poisson arrivals, served frames)" if srv else None},
            "parity": parity,
            "roofline": roofline,
            "legs": legs or None,
            "with_residuals": with_residuals,
            "smoother": smoother,
            "rans": codec,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(tm["kernel_launches"]) * args.steps,
            "clocks": clk,
            "kernel_ms": {"prepare": tm["prepare_ms_sum"] / tm["n_timed"], "sort": tm["sort_ms_sum"] / tm["n_timed"],
                          "fit": tm["fit_ms_sum"] / tm["n_timed"], "sequence": tm["total_ms_sum"] / tm["n_timed"]},
        }
        print(json.dumps(line), flush=True)
    fx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
