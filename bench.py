#!/usr/bin/env python
"""Cell-graph build throughput on one scene per GPU.

Workload: l = 64 planes in 3-space (a in [-1024,1024]^3, b in [-2^30,2^30]),
N = 2^24 integer points in [-2^20,2^20]^3 (seeded, synthetic). One step = the
whole hot path on that scene (exact sign vectors, duplicate removal into sorted
cells, Hamming-1 search and edge compaction) through cg_build_dev, whose last
kernel writes U, E and a status on the device, followed by an asynchronous
copy of those counts to pinned host memory; the K timed steps are enqueued back
to back (no host wait between them) and every step's counts are checked after
the timed region. The same builds as synchronous cg_build calls (counts read
back before each call returns) are reported beside it (``sync_call_ms``), and
``e2e`` times the host-buffer call cg_build_host.

Prints one JSON line (rank 0). ``--impl reference`` times the plain CPU oracle
on a bounded sample of the same workload instead.

Multi-GPU: one process per GPU (torchrun); every rank builds its own replica
scene (no data exchange: scenes are independent units), ``value`` is the
points all ranks processed per second over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The batch overlaps scenes on 32 worker streams; let them map to as many
# hardware work queues (read when the CUDA context is created).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = ("cell-graph build Mvectors/s (dedup+Hamming-1 edges), %HBM peak; batched vs plain")
UNIT = "Mvectors/s"
N_POINTS = 1 << 24
ELL = 64
DIM = 3
WORKLOAD = "planes_3d: l=64 planes, d=3, N=2^24 int32 points in [-2^20,2^20]^3"

# DRAM bytes (read + write) of one launch of each fused sign+dedup kernel from
# an ncu capture, with the digest of the kernel source's code (sha256 of the
# file with comments and white space removed) they were taken on; reported
# only while that code is unchanged.
NCU_TRAFFIC = {
    "code_sha256": "f605913e787c8f673387b032aafdb6a3b6bb61683be055010e5447656fbd9a2d",
    "bytes_per_launch": {"pack_fast_kernel": 205276416.0, "pack_grid_kernel": 220094976.0},
}


def code_digest(path: str) -> str:
    """sha256 of a C++/CUDA source with its comments and white space removed."""
    src = open(path, encoding="utf-8").read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return hashlib.sha256(" ".join(src.split()).encode()).hexdigest()

# SHA-256 digests of the CPU oracle's complete outputs on the full-size
# workloads, written by a script that calls only the oracle.
DIGESTS = os.path.join(ROOT, "tests", "golden", "full_size_digests.json")


def golden_digests() -> dict:
    with open(DIGESTS) as f:
        return json.load(f)


def digest_of(arr) -> str:
    """SHA-256 of an array's bytes (a CUDA tensor is copied to the host)."""
    import numpy as np

    if hasattr(arr, "cpu"):
        arr = arr.cpu().numpy()
    return hashlib.sha256(np.ascontiguousarray(arr).tobytes()).hexdigest()


def digest_mismatch(entry: dict, cells, edges) -> bool:
    return (cells.shape[0] != entry["n_cells"] or edges.shape[0] != entry["n_edges"]
            or digest_of(cells) != entry["cells_sha256"]
            or digest_of(edges) != entry["edges_sha256"])


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """Samples SM clocks and clock-event (throttle) reasons while the timed
    region runs: NVML through ctypes every ~2 ms (the timed region can be a few
    ms long), plus nvidia-smi at 200 ms when the region is long enough."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    SMI_FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                  "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, cuda_index: int):
        self.cuda_index = cuda_index
        self.sm, self.reason_bits, self.max_mhz = [], 0, None
        self.smi_lines = []
        self._stop = threading.Event()
        self._nvml = None
        self._handle = None

    def _nvml_open(self):
        import ctypes

        import torch

        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return False
        h = ctypes.c_void_p()
        uuid = "GPU-" + str(torch.cuda.get_device_properties(self.cuda_index).uuid)
        if lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) != 0:
            if lib.nvmlDeviceGetHandleByIndex_v2(self.cuda_index, ctypes.byref(h)) != 0:
                return False
        self._nvml, self._handle = lib, h
        v = ctypes.c_uint(0)
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(v)) == 0:
            self.max_mhz = float(v.value)
        return True

    def _poll(self):
        import ctypes

        lib, h = self._nvml, self._handle
        v = ctypes.c_uint(0)
        r = ctypes.c_ulonglong(0)
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or getattr(
            lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(v)) == 0:
                self.sm.append(float(v.value))
            if get_reasons(h, ctypes.byref(r)) == 0:
                self.reason_bits |= int(r.value)
            time.sleep(0.002)

    def _smi(self):
        for line in self._proc.stdout:
            self.smi_lines.append(line.strip())

    def __enter__(self):
        self._threads = []
        try:
            if self._nvml_open():
                t = threading.Thread(target=self._poll, daemon=True)
                t.start()
                self._threads.append(t)
        except Exception:
            self._nvml = None
        self._proc = None
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.SMI_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            t = threading.Thread(target=self._smi, daemon=True)
            t.start()
            self._threads.append(t)
        except Exception:
            self._proc = None
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        for t in self._threads:
            t.join(timeout=5)

    def summary(self):
        reasons = {name for bit, name in self.REASONS.items() if self.reason_bits & bit}
        sm = list(self.sm)
        for ln in self.smi_lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                self.max_mhz = max(self.max_mhz or 0.0, float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"], parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"],
                    "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(sm),
                "nvidia_smi_samples": len(self.smi_lines)}


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Largest x over all ranks of the process group (x itself without one)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_rank: int, seconds: float) -> float:
    """Whole-job throughput in millions of units per second: every rank
    processes units_per_rank, the job takes the slowest rank's seconds."""
    return world * units_per_rank / seconds / 1e6


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_description() -> dict:
    """The host the CPU baseline ran on: architecture, CPU model (from
    /proc/cpuinfo where it has one) and logical core count."""
    import platform

    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key, _, val = line.partition(":")
                key = key.strip().lower()
                if key in ("model name", "cpu model", "hardware") and val.strip():
                    model = val.strip()
                    break
                if key == "cpu part" and model is None:
                    model = f"cpu part {val.strip()}"
    except OSError:
        pass
    return {"machine": platform.machine(), "model": model or platform.processor() or None,
            "logical_cores": os.cpu_count()}


def cpu_baseline(sample_points: int, seed: int = 2):
    """Times the CPU oracle (single thread) on the first ``sample_points``
    points of the workload."""
    import oracle
    from paper_1503_06029_gb300 import inputs

    sc = inputs.planes_3d(n=N_POINTS, ell=ELL, seed=seed)
    pts = sc.pts[:sample_points].copy()
    oracle.compile_library()
    t0 = time.perf_counter()
    cells, edges = oracle.build(pts, sc.a, sc.b, 64)
    dt = time.perf_counter() - t0
    return {"value": sample_points / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {sample_points} points of the workload scene "
                      f"({len(cells)} cells, {len(edges)} edges), {dt:.2f} s single-threaded",
            "host": host_description()}


def batch_compare(ctx, dev, steps: int):
    """The batched workload: 1,024 independent 3-D scenes, l log-uniform in
    [8, 256] (multiple of 8), N log-uniform in [1e3, 1e6], all resident. Times
    one cg_build_batch call per step against one pass of plain cg_build calls
    over the same scenes on the same GPU."""
    import torch

    from paper_1503_06029_gb300 import cellgraph, inputs

    spec = inputs.scene_batch_spec()
    scenes = []
    for s in range(len(spec.n)):
        sc = inputs.batch_scene(spec, s)
        scenes.append((torch.from_numpy(sc.pts).to(dev), torch.from_numpy(sc.a).to(dev),
                       torch.from_numpy(sc.b).to(dev)))
    total = int(spec.n.sum())
    stream = torch.cuda.current_stream()
    t_tune = time.perf_counter()
    tuned = ctx.autotune(scenes, reps=1)
    t_tune = time.perf_counter() - t_tune
    for _ in range(3):  # sizes learned, then captured, then replayed
        res = ctx.build_batch(scenes)
    cells = sum(int(c.shape[0]) for c, _ in res)
    edges = sum(int(e.shape[0]) for _, e in res)
    # Compulsory bytes: each scene's points read once (4 d B each), its cells
    # (8 W B each) and edges (8 B each) written once.
    compulsory = sum(4.0 * int(pts.shape[1]) * int(pts.shape[0]) +
                     8.0 * ((int(a.shape[0]) + 63) // 64) * int(c.shape[0]) + 8.0 * int(e.shape[0])
                     for (pts, a, _), (c, e) in zip(scenes, res))
    launches0 = cg_launches()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(steps):
        ctx.build_batch(scenes, as_views=False)
    t1.record(stream)
    torch.cuda.synchronize()
    batch_ms = t0.elapsed_time(t1) / steps
    batch_launches = (cg_launches() - launches0) // steps
    outs = []
    for pts, a, b in scenes:
        c, e = ctx.build(pts, a, b, 64)
        outs.append((torch.empty_like(c), torch.empty_like(e)))
    passes = max(1, steps // 4)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(passes):
        for (pts, a, b), o in zip(scenes, outs):
            ctx.build(pts, a, b, 64, outputs=o)
    t1.record(stream)
    torch.cuda.synchronize()
    plain_ms = t0.elapsed_time(t1) / passes
    # Every scene of the replayed batch against the oracle's digests.
    entries = golden_digests()["batch_scenes"]
    res = ctx.build_batch(scenes)
    bad = sum(digest_mismatch(entries[i], c, e) for i, (c, e) in enumerate(res))
    return {"workload": "1,024 scenes, l in [8,256], N in [1e3,1e6] log-uniform, d=3",
            "points": total, "cells": cells, "edges": edges,
            "oracle_digest_mismatches": int(bad),
            "batched": {"value": total / (batch_ms * 1e-3) / 1e6, "unit": UNIT,
                        "ms_per_batch": batch_ms, "gpu_launches_per_batch": batch_launches,
                        "compulsory_bytes": compulsory,
                        "hbm_frac": compulsory / (batch_ms * 1e-3) / 1e9 / _hbm_peak_gbs()},
            "plain": {"value": total / (plain_ms * 1e-3) / 1e6, "unit": UNIT,
                      "ms_per_batch": plain_ms, "calls": len(scenes)},
            "speedup": plain_ms / batch_ms,
            "autotune": {"seconds": t_tune,
                         "chosen": {str(cellgraph.TUNE_LIMITS[b]): v["setting"]
                                    for b, v in tuned.items()}}}


def serve_measure(dev, capacity_scenes_per_s: float, n_requests: int = 2000,
                  loads=(0.25, 0.5, 0.9), pool_scenes: int = 256, tuned_ctx=None):
    """Serving: Poisson arrivals (exponential gaps, seed 5) of scenes drawn as
    in the batched workload, offered at fractions of the measured batched
    capacity (scenes/s). Requests go through the request server with host
    inputs in pinned memory (copied by the server after admission). When a
    level's submissions are done, each request is waited for in arrival
    order; once all have finished, each one's cells and edges are fetched,
    their SHA-256 digests compared with the oracle's for the same scene, and
    the request is released (the budget holds every result of a level, so
    admission never waits for a release; keeping the Python client off the
    interpreter lock while submitting is what lets the offered rate be met).
    Latency = completion on the device (server stamp) minus submission on the
    host (server stamp)."""
    import numpy as np
    import torch

    from paper_1503_06029_gb300 import cellgraph, inputs

    spec = inputs.scene_batch_spec()
    pool = []
    for s in range(pool_scenes):
        sc = inputs.batch_scene(spec, s)
        pool.append(tuple(torch.from_numpy(x).pin_memory().numpy() for x in (sc.pts, sc.a, sc.b)))
    want = golden_digests()["batch_scenes"]  # the oracle's outputs of these scenes
    out = {"workload": "Poisson stream of scenes drawn like the batched workload "
                       f"(a pool of {pool_scenes} scenes, cycled), host inputs in pinned memory",
           "capacity_scenes_per_s": capacity_scenes_per_s, "levels": []}
    with cellgraph.Server(dev.index or 0, hbm_budget_bytes=16 << 30, max_inflight=32) as srv:
        if tuned_ctx is not None:
            srv.use_tuning(tuned_ctx)
        for k in range(32):  # warm-up: kernels loaded, pool memory cached
            t = srv.submit(*pool[k % pool_scenes])
            srv.wait(t)
            srv.release(t)
        for load in loads:
            rate = load * capacity_scenes_per_s
            arrivals = inputs.poisson_arrivals(n_requests, rate, seed=5)
            tickets = [None] * n_requests
            lat, mism = [], [0]
            first_submit, last_done = [None], [0.0]
            t0 = time.perf_counter()
            for i in range(n_requests):
                gap = arrivals[i] - (time.perf_counter() - t0)
                if gap > 3e-4:
                    time.sleep(gap - 2e-4)
                while time.perf_counter() - t0 < arrivals[i]:
                    pass
                tickets[i] = srv.submit(*pool[i % pool_scenes])
            for i in range(n_requests):
                srv.wait(tickets[i])
                r = srv.result(tickets[i])
                mism[0] += int(r["status"] != 0)
                lat.append(r["done_us"] - r["submit_us"])
                if first_submit[0] is None:
                    first_submit[0] = r["submit_us"]
                last_done[0] = max(last_done[0], r["done_us"])
            # Once every request of the level has finished (the budget holds all
            # results), each one's cells and edges against the oracle's digests.
            for i in range(n_requests):
                if srv.result(tickets[i])["status"] == 0:
                    cells, edges = srv.fetch(tickets[i])
                    mism[0] += digest_mismatch(want[i % pool_scenes], cells, edges)
                srv.release(tickets[i])
            pts_total = sum(int(pool[i % pool_scenes][0].shape[0]) for i in range(n_requests))
            span_s = (last_done[0] - first_submit[0]) * 1e-6
            st = srv.stats()
            lat_ms = np.array(lat) * 1e-3
            out["levels"].append({
                "offered_load": load, "offered_scenes_per_s": rate, "requests": n_requests,
                "p50_ms": float(np.percentile(lat_ms, 50)),
                "p99_ms": float(np.percentile(lat_ms, 99)),
                "mean_ms": float(lat_ms.mean()),
                "sustained": {"value": pts_total / span_s / 1e6, "unit": UNIT,
                              "scenes_per_s": n_requests / span_s},
                "oracle_digest_mismatches": mism[0], "max_running": st["max_running"],
                "peak_bytes": st["peak_bytes"], "groups_so_far": st["groups"],
                "grouped_so_far": st["grouped"]})
    return out


def chains_measure(dev, steps: int, strategies=("hash", "pivot", "tree", "halves")):
    """Long vectors: l = 1024 (16 words), 2^18 random seeds with 15-step
    single-flip chains, 25% duplicated, N = 5,242,880 vectors resident on the
    device. One step = cg_dedup_cells + cg_neighbors_h1 (counts read back),
    per lookup strategy of the neighbour search."""
    import numpy as np
    import torch

    from paper_1503_06029_gb300 import cellgraph, inputs

    ch = inputs.chains()
    n = int(ch.keys.shape[0])
    keys = torch.from_numpy(ch.keys.view(np.int64)).to(dev)
    del ch
    out = {"workload": "chains: l=1024 (16 x uint64), 2^18 seeds x 16 chain members + 25% "
                       "duplicates, N=5,242,880", "n": n, "strategies": {}}
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for strat in strategies:
        for _ in range(2):
            cells = cellgraph.dedup_cells(keys, 1024, 64)
            edges = cellgraph.neighbors_h1(cells, 1024, 64, strategy=strat)
        d_ms = n_ms = 0.0
        for _ in range(steps):
            ev[0].record(stream)
            cells = cellgraph.dedup_cells(keys, 1024, 64)
            ev[1].record(stream)
            edges = cellgraph.neighbors_h1(cells, 1024, 64, strategy=strat)
            ev[2].record(stream)
            torch.cuda.synchronize()
            d_ms += ev[0].elapsed_time(ev[1]) / steps
            n_ms += ev[1].elapsed_time(ev[2]) / steps
        out["cells"], out["edges"] = int(cells.shape[0]), int(edges.shape[0])
        # Compulsory bytes: the vectors read once, the cells and edges written once.
        compulsory = 128.0 * n + 128.0 * out["cells"] + 8.0 * out["edges"]
        out["compulsory_bytes"] = compulsory
        out["strategies"][strat] = {"value": n / ((d_ms + n_ms) * 1e-3) / 1e6, "unit": UNIT,
                                    "ms_per_step": d_ms + n_ms, "dedup_ms": d_ms,
                                    "neighbors_ms": n_ms,
                                    "hbm_frac": compulsory / ((d_ms + n_ms) * 1e-3) / 1e9 /
                                    _hbm_peak_gbs()}
    return out


def _hbm_peak_gbs() -> float:
    """Measured HBM copy rate (MEASURED_PEAKS.json), GB/s."""
    peaks, _ = _peaks()
    return float(peaks.get("hbm_gbs", 6800.0))


def _alu_peak_tmacs() -> float:
    """FP32 lane peak in T multiply-adds/s: 152 SMs x 128 lanes x the
    measured maximum SM clock (MEASURED_PEAKS.json), one MAC per lane-FMA."""
    peaks, _ = _peaks()
    return 152 * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def quadric_measure(dev, steps: int):
    """Curved boundaries: l = 64 spheres in 3-space (the quadric form of
    |p - c_i|^2 >= r_i^2), N = 2^24 points, device-resident. One step =
    cg_pack_signs_quadric + cg_dedup_cells + cg_neighbors_h1 (the last two read
    their counts back). Reports Mvectors/s, the quadric sign kernel's time and
    its fraction of the FP32 lane peak (N l F multiply-adds, F = 9 features:
    six monomials and three coordinates), and checks the output against the
    oracle's digest when one is stored."""
    import torch

    from paper_1503_06029_gb300 import cellgraph, inputs

    sc = inputs.spheres_3d()
    n, ell = sc.n, sc.ell
    t = [torch.from_numpy(x).to(dev) for x in (sc.pts, sc.q, sc.a, sc.b)]
    del sc
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(2):
        cells, edges = cellgraph.build_quadric(*t, 64)
    pack_ms = step_ms = 0.0
    for _ in range(steps):
        ev[0].record(stream)
        keys = cellgraph.pack_signs_quadric(*t, 64)
        ev[1].record(stream)
        cells = cellgraph.dedup_cells(keys, ell, 64)
        edges = cellgraph.neighbors_h1(cells, ell, 64)
        ev[2].record(stream)
        torch.cuda.synchronize()
        pack_ms += ev[0].elapsed_time(ev[1]) / steps
        step_ms += ev[0].elapsed_time(ev[2]) / steps
    peak = _alu_peak_tmacs()
    work = float(n) * ell * 9
    out = {"workload": "spheres_3d: l=64 spheres (quadrics), d=3, N=2^24 int32 points in "
                       "[-2^20,2^20]^3, radii in [2^19,2^21]",
           "value": n / (step_ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": step_ms,
           "cells": int(cells.shape[0]), "edges": int(edges.shape[0]),
           "sign_kernel": {"ms": pack_ms, "achieved": work / (pack_ms * 1e-3) / 1e12,
                           "peak": peak, "unit": "TMAC/s",
                           "frac": work / (pack_ms * 1e-3) / 1e12 / peak,
                           "work": "N*l*F exact multiply-adds, F = 9"}}
    entry = golden_digests().get("spheres_3d")
    if entry is not None:
        out["oracle_digest_mismatch"] = bool(digest_mismatch(entry, cells, edges))
    return out


def bfs_measure(ctx, dev, steps: int):
    """Breadth-first search on a cell graph (paths in G_X, §6): the graph of
    l = 256 planes in 3-space over 2^22 points (drawn like planes_3d), built
    once; one step = cg_bfs from cell 0 (adjacency build + levels, distances
    and parents), timed with CUDA events."""
    import torch

    from paper_1503_06029_gb300 import cellgraph, inputs

    sc = inputs.planes_3d(n=1 << 22, ell=256, seed=12)
    cells, edges = ctx.build(*(torch.from_numpy(x).to(dev) for x in (sc.pts, sc.a, sc.b)), 64)
    u, e = int(cells.shape[0]), int(edges.shape[0])
    for _ in range(2):
        dist, par, reached, depth = cellgraph.bfs(edges, u, 0)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ms = []
    for _ in range(steps):
        ev[0].record(stream)
        dist, par, reached, depth = cellgraph.bfs(edges, u, 0)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms.append(ev[0].elapsed_time(ev[1]))
    t = statistics.median(ms)
    ed = edges.long()
    comp = int(((dist[ed[:, 0]] >= 0) & (dist[ed[:, 1]] >= 0)).sum())  # edges searched
    return {"workload": "cell graph of l=256 planes in 3-space over 2^22 points (like planes_3d), "
                        "BFS from cell 0 with parents", "cells": u, "edges": e,
            "reached": reached, "component_edges": comp, "depth": depth, "ms": t,
            "value": comp / (t * 1e-3) / 1e6,
            "unit": "Medges/s (undirected edges of the source's component per second)"}


def inputs_spec_n():
    from paper_1503_06029_gb300 import inputs

    return inputs.scene_batch_spec().n


def cg_launches():
    from paper_1503_06029_gb300 import cellgraph

    return cellgraph.launch_count()


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_1503_06029_gb300 import inputs

    oracle.compile_library()
    sc = inputs.planes_3d(n=N_POINTS, ell=ELL, seed=2)
    sample = args.ref_sample
    times = []
    for step in range(args.warmup + args.steps):
        lo = (step * sample) % (N_POINTS - sample + 1)
        pts = sc.pts[lo: lo + sample].copy()
        t0 = time.perf_counter()
        oracle.build(pts, sc.a, sc.b, 64)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_step = sum(times) / len(times)
    value = sample / per_step / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{sample} consecutive points of the workload scene per step",
                         "host": host_description()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if pg:
        pg.barrier()
    from paper_1503_06029_gb300 import cellgraph, inputs

    n = args.n
    sc = inputs.planes_3d(n=n, ell=ELL, seed=2 + rank)
    pts = torch.from_numpy(sc.pts).to(dev)
    a = torch.from_numpy(sc.a).to(dev)
    b = torch.from_numpy(sc.b).to(dev)
    ctx = cellgraph.Context(local)
    if args.sign_kernel >= 0:  # one sign kernel for every bucket of l
        for bucket in range(cellgraph.TUNE_BUCKETS):
            t = ctx.tune_get(bucket)
            ctx.tune_set(bucket, t["strategy"], t["pivots"], args.sign_kernel)
    cells, edges = ctx.build(pts, a, b, 64)  # sizes the outputs
    u, e = cells.shape[0], edges.shape[0]
    outputs = (torch.empty((u, 1), dtype=torch.int64, device=dev),
               torch.empty((e, 2), dtype=torch.int32, device=dev))
    # Buffers of the timed builds: cg_build_dev writes U, E and a status to a
    # device word triple, copied to pinned host memory after every step.
    dev_cells = torch.empty((u + 64, 1), dtype=torch.int64, device=dev)
    dev_edges = torch.empty((e + 64, 2), dtype=torch.int32, device=dev)
    dev_counts = torch.zeros(3, dtype=torch.int64, device=dev)
    host_counts = torch.zeros((args.steps, 3), dtype=torch.int64).pin_memory()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctx.build(pts, a, b, 64, outputs=outputs)  # also settles the table size
        ctx.build_dev(pts, a, b, dev_cells, dev_edges, dev_counts)
    torch.cuda.synchronize()

    # ---- device-resident timed region: K whole builds enqueued back to back,
    # each step's counts copied back to the host without a wait ----
    launches0 = cellgraph.launch_count()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        start.record(stream)
        for k in range(args.steps):
            ctx.build_dev(pts, a, b, dev_cells, dev_edges, dev_counts)
            host_counts[k].copy_(dev_counts, non_blocking=True)
        stop.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
    launches = cellgraph.launch_count() - launches0
    ms = max_over_ranks(start.elapsed_time(stop) / args.steps, pg, dev)
    bad = [k for k in range(args.steps) if host_counts[k].tolist() != [u, e, 0]]
    if bad:
        raise RuntimeError(f"timed build {bad[0]} returned counts {host_counts[bad[0]].tolist()}, "
                           f"expected {[u, e, 0]}")
    # The same builds one synchronous call at a time (counts read back before
    # each call returns), for reference.
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(args.steps):
        ctx.build(pts, a, b, 64, outputs=outputs)
    stop.record(stream)
    torch.cuda.synchronize()
    sync_ms = max_over_ranks(start.elapsed_time(stop) / args.steps, pg, dev)
    # Stage split from a separate pass (the stage timers record CUDA events
    # between the stages and turn off the graph replay of repeated builds).
    ctx.set_timing(True)
    for _ in range(args.steps):
        ctx.build(pts, a, b, 64, outputs=outputs)
    torch.cuda.synchronize()
    stages, builds = ctx.stage_times()
    ctx.set_timing(False)
    value = job_value(world, n, ms * 1e-3)

    # ---- end to end through the C-ABI with host buffers ----
    pin = lambda x: torch.from_numpy(x).pin_memory().numpy()
    h_pts, h_a, h_b = pin(sc.pts), pin(sc.a), pin(sc.b)
    h_out = (torch.empty((u, 1), dtype=torch.int64).pin_memory().numpy().view(np.uint64),
             torch.empty((e, 2), dtype=torch.int32).pin_memory().numpy().view(np.uint32))
    for _ in range(2):
        ctx.build_host(h_pts, h_a, h_b, 64, outputs=h_out)
    e2e_steps = max(3, args.steps // 2)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        hc, he = ctx.build_host(h_pts, h_a, h_b, 64, outputs=h_out)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, pg, dev)
    h2d = sc.pts.nbytes + sc.a.nbytes + sc.b.nbytes
    d2h = hc.nbytes + he.nbytes

    peaks, peak_kind = _peaks()
    # Dominant kernel: the sign step (stage "pack_dedup"). With the box grid
    # (stage "grid" before it) it is the fused sign + dedup kernel that tests
    # each point against its grid cell's crossing constraints only: bound by
    # reading the points (12 B each) from HBM. Without it, every constraint is
    # tested per point: N*l*d multiply-adds on the FP32 lanes.
    k_ms = stages.get("pack_dedup", float("nan")) / max(1, builds)
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    same_source = NCU_TRAFFIC["code_sha256"] == code_digest(
        os.path.join(ROOT, "paper_1503_06029_gb300", "csrc", "cg_pack.cu"))
    traffic = {k: (v if same_source else None)
               for k, v in NCU_TRAFFIC["bytes_per_launch"].items()}
    timing_note = ("CUDA events between the build's stages on its stream, in a second pass "
                   "of the same builds")
    if "grid" in stages:
        alg = 12.0 * n
        achieved = alg / (k_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm",
                    "kernel": "pack_grid_kernel<3, 2, FastInsert> (sign + dedup on the box grid)",
                    "grid_setup_ms": stages.get("grid", float("nan")) / max(1, builds),
                    "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": traffic["pack_grid_kernel"],
                    "peak_note": f"HBM copy rate ({peak_kind})", "kernel_ms": k_ms,
                    "work": "12 B of int32 coordinates read per point (N points per launch)",
                    "kernel_timing": timing_note}
    else:
        macs = float(n) * ELL * DIM
        alu_peak = 152 * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12  # TMAC/s
        achieved = macs / (k_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": "pack_fast_kernel<3, 2, FastInsert> (sign + dedup)",
                    "achieved": achieved, "peak": alu_peak, "unit": "TMAC/s",
                    "frac": achieved / alu_peak, "traffic": traffic["pack_fast_kernel"],
                    "peak_note": f"152 SMs x 128 FP32 lanes x {peaks.get('sm_max_mhz')} MHz "
                                 f"({peak_kind} max clock); one MAC = one lane-FMA",
                    "kernel_ms": k_ms, "work": "N*l*d exact multiply-adds",
                    "kernel_timing": timing_note}
    compulsory = 12.0 * n + 8.0 * u + 8.0 * e
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_points": n, "ell": ELL, "d": DIM, "cells": u,
                   "edges": e, "l2": "inputs larger than L2 (201 MB of points per step)",
                   "replicas": world,
                   "timing": "K cg_build_dev steps enqueued back to back, each step's counts "
                             "copied to pinned host memory without a wait and all checked "
                             "after the timed region"},
        "sync_call_ms": sync_ms,
        "roofline": roofline,
        "hbm_step": {"compulsory_bytes": compulsory,
                     "achieved_gbs": compulsory / (ms * 1e-3) / 1e9,
                     "peak_gbs": hbm_peak,
                     "frac": compulsory / (ms * 1e-3) / 1e9 / hbm_peak,
                     "peak_kind": peak_kind},
        "stages_ms": {k: v / max(1, builds) for k, v in stages.items()},
        "e2e": {"value": job_value(world, n, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    # Batch and serving first: the server's host threads measured slower (and
    # more variable) after the long-vector section had run in the process.
    if not args.no_batch:
        line["batch"] = batch_compare(ctx, dev, max(3, args.steps // 2))
        if not args.no_serve:
            cap = len(inputs_spec_n()) / (line["batch"]["batched"]["ms_per_batch"] * 1e-3)
            line["serve"] = serve_measure(dev, cap, n_requests=args.serve_requests,
                                          tuned_ctx=ctx)
    if not args.no_chains:
        line["chains"] = chains_measure(dev, max(3, args.steps // 4),
                                        tuple(args.chains_strategies.split(",")))
    if not args.no_bfs:
        line["bfs"] = bfs_measure(ctx, dev, max(5, args.steps // 2))
    if not args.no_quadric:
        line["quadric"] = quadric_measure(dev, max(5, args.steps // 2))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=N_POINTS)
    p.add_argument("--cpu-sample", type=int, default=1 << 24)
    p.add_argument("--ref-sample", type=int, default=1 << 20)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--sign-kernel", type=int, default=-1,
                   help="headline builds with this tuning sign_kernel (0 fp32 default, 1 tensor "
                        "cores, 2 box grid, 3 all constraints); -1: the library default")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the batched-vs-plain comparison (and serving)")
    p.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    p.add_argument("--no-chains", action="store_true", help="skip the long-vector workload")
    p.add_argument("--no-bfs", action="store_true", help="skip the BFS measurement")
    p.add_argument("--no-quadric", action="store_true",
                   help="skip the quadric-constraint (spheres) measurement")
    p.add_argument("--chains-strategies", default="hash,pivot,tree,halves",
                   help="lookup strategies timed on the long-vector workload")
    p.add_argument("--serve-requests", type=int, default=2000)
    args = p.parse_args()
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
