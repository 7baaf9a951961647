#!/usr/bin/env python
"""Benchmark of the muon g-2 waveform DAQ hot path (T-method islands + Q-method histograms).

Default workload: one full fill, 24 calorimeters x 54 crystals x 560,000 int16
samples (1.4515 GB), seeded synthetic waveforms, device-resident.  A step is
one pass of the whole path over the fill: pedestals, crystal sum, threshold,
pre/post windows, merge, island records + pool rows, Q decimation and the
int64 fill-by-fill sum.  The input (1.45 GB) is larger than L2 (129 MB), so
no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  Under torchrun each rank processes its own fill
on its own GPU (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import ctypes
import glob
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

METRIC = "raw waveform GB/s (T+Q) and % of HBM peak; p99 per-fill latency"
UNIT = "GB/s"
NOMINAL_HBM_GBS = 7900.0


# ----------------------------------------------------------------------------- helpers
def measured_peaks() -> tuple:
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Sources compiled into the two-pass kernels (prepare, count, scan, compact).
KERNEL_SOURCES = ("daq_device.cuh", "daq_steps.cuh", "daq_twopass.cuh", "daq_process.cu")


def kernel_source_hash() -> str:
    """Hash of the code (comments and whitespace left out, so that editing a
    comment does not void a profile taken on the same kernels)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        text = open(os.path.join(ROOT, "paper_1611_04959_gb300", "csrc", name), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    fn = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    if not os.path.exists(fn):
        return None
    kv = {}
    for line in open(fn):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256") != kernel_source_hash():
        return None
    try:
        return float(kv["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """Samples SM clock and clock-event reasons through NVML (read-only) while
    the timed region runs; falls back to `nvidia-smi -lms`."""
    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
               0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}

    def __init__(self, index: int, period_s: float = 0.01):
        self.index, self.period = index, period_s
        self.samples, self.max_mhz, self._stop = [], None, threading.Event()
        self._nvml = None
        self._proc = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() == 0:
                h = ctypes.c_void_p()
                if nv.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(h)) == 0:
                    self._nvml, self._h = nv, h
                    mx = ctypes.c_uint()
                    if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
                        self.max_mhz = int(mx.value)
        except OSError:
            self._nvml = None

    def _run(self):
        nv, h = self._nvml, self._h
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        get_r = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._stop.is_set():
            if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and get_r(h, ctypes.byref(rs)) == 0:
                self.samples.append((int(clk.value), int(rs.value)))
            time.sleep(self.period)

    def __enter__(self):
        if self._nvml is not None:
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        else:
            q = ("index,clocks.sm,clocks.max.sm,clocks_event_reasons.active")
            self._proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                           "--format=csv,noheader,nounits", "-lms", "100"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        return self

    def __exit__(self, *exc):
        if self._nvml is not None:
            self._stop.set()
            self._t.join()
        elif self._proc is not None:
            self._proc.terminate()
            out, _ = self._proc.communicate(timeout=10)
            for line in out.splitlines():
                try:
                    _, sm, mx, act = [v.strip() for v in line.split(",")]
                    self.samples.append((int(sm), int(act, 16)))
                    self.max_mhz = int(mx)
                except ValueError:
                    pass

    def summary(self) -> dict:
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0}
        bits = 0
        for _, r in self.samples:
            bits |= r
        names = [n for b, n in self.REASONS.items() if bits & b and n != "gpu_idle"]
        return {"sm_mhz": statistics.median(s for s, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": names, "samples": len(self.samples)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- CPU baseline (oracle)
def run_cpu_oracle(samples_np, params, target_s: float, calos: int | None = None, length: int | None = None,
                   threads: int | None = None):
    """Time the oracle, as it stands, on a bounded sample of the workload:
    the first `calos` calorimeters x `length` samples, repeated until
    target_s of CPU work, on `threads` host threads (default: all cores).
    Returns (GB/s, seconds, repeats, threads, bytes)."""
    import numpy as np
    import oracle
    F, C, X, N = samples_np.shape
    calos = calos or C
    length = length or N
    sub = np.ascontiguousarray(samples_np[:1, :calos, :, :length])
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.process_fills(sub, params, n_threads=threads)
        reps += 1
        if time.perf_counter() - t0 >= target_s:
            break
    dt = time.perf_counter() - t0
    return reps * sub.nbytes / dt / 1e9, dt, reps, threads, sub.nbytes


# ----------------------------------------------------------------------------- GB300 arm
def bench_gb300(args, ws, rank, local):
    import numpy as np
    import torch

    import synth
    import paper_1611_04959_gb300 as daq
    from paper_1611_04959_gb300 import build as daq_build
    from paper_1611_04959_gb300 import replicas
    from synth import workloads as W

    daq_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w = W.PLAIN_FULL_FILL if args.calos == 24 else W.scaled(W.PLAIN_FULL_FILL, n_calo=args.calos)
    params = w.params()
    F, C, X, N = w.n_fills, w.n_calo, 54, w.n_samples
    host = torch.empty((F, C, X, N), dtype=torch.int16).pin_memory()
    # rank r processes fill r of the generator (its own share; weak scaling)
    synth.generate(W.scaled(w, n_fills=max(1, ws)).config(), out=host.numpy(), n_threads=os.cpu_count() or 1,
                   fills=(rank, 1))
    samples = host.to(dev)
    raw_bytes = samples.numel() * 2

    stream = torch.cuda.Stream(dev)
    rows_cap = F * C * N
    out = daq.Outputs(torch, dev, F, C, X, rows_cap // 2 + F * C + 1, rows_cap)
    q = torch.zeros(daq.q_size(C, N, params["decim"]), dtype=torch.int64, device=dev)

    def make_p(grid=0):
        p = daq.make_params(**params, stream=stream, grid=grid)
        nbytes = daq.daq_workspace_size(C, X, N, F, p)
        return p, nbytes

    p, wsb = make_p()
    workspace = torch.empty(wsb, dtype=torch.uint8, device=dev)
    p.workspace, p.workspace_bytes = workspace.data_ptr(), wsb
    isl = out.struct()

    def call(pp, ev_ptrs=None):
        pp.events = ev_ptrs
        rc = daq.daq_process_fills(samples.data_ptr(), C, X, N, F, pp, isl, q.data_ptr())
        if rc != daq.DAQ_OK:
            raise daq.DaqError(rc, "daq_process_fills")

    def barrier():
        torch.cuda.synchronize(dev)
        replicas.barrier(dev)
        torch.cuda.synchronize(dev)

    # ---- warm-up
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            call(p)
    torch.cuda.synchronize(dev)
    counts = out.counts.cpu().numpy()
    status = daq.daq_status_from_counts(counts)
    if status != daq.DAQ_OK:
        raise daq.DaqError(status, "warm-up")
    n_isl, n_rows = int(counts[0]), int(counts[1])

    # ---- timed region: K steps bracketed by two events, nothing else on the stream
    K = args.steps
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clocks:
        with torch.cuda.stream(stream):
            t_start.record(stream)
            for _ in range(K):
                call(p)
            t_end.record(stream)
        torch.cuda.synchronize(dev)
    elapsed_ms = t_start.elapsed_time(t_end)

    # ---- per-kernel times and per-step latency: a second run with DAQ_N_EVENTS events per step
    # [0] start, [1] after pedestals, [2] after count kernel, [3] after scan, [4] end
    # (the events cost about 10 us per step, so they stay out of the timed region)
    Kd = max(3, min(K, 500))
    NE = 5
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(NE)] for _ in range(Kd)]
    for trio in evs:                      # creates the events before their handles are taken
        for e in trio:
            e.record(stream)
    ev_arrays = [(ctypes.c_void_p * NE)(*[e.cuda_event for e in trio]) for trio in evs]
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for k in range(Kd):
            call(p, ctypes.cast(ev_arrays[k], ctypes.c_void_p).value)
    torch.cuda.synchronize(dev)
    step_ms = [e[0].elapsed_time(e[4]) for e in evs]
    prep_ms = [e[0].elapsed_time(e[1]) for e in evs]
    count_ms = [e[1].elapsed_time(e[2]) for e in evs]
    scan_ms = [e[2].elapsed_time(e[3]) for e in evs]
    compact_ms = [e[3].elapsed_time(e[4]) for e in evs]
    _, elapsed_ms, value = replicas.aggregate(K * raw_bytes, elapsed_ms, dev)

    # ---- roofline of the dominant kernel: the compact pass (reads the samples, writes the islands)
    peak, peak_kind = measured_peaks()
    q_bytes = sum(C * daq.daq_q_bins(N, d) * 16 for d in params["decim"])
    n_tiles = F * C * (-(-N // 448))
    side = n_tiles * (14 * 4 + 16 + 16)             # marks words, aggregate, prefix per tile
    alg_count = raw_bytes + q_bytes + side
    alg_compact = raw_bytes + n_rows * X * 2 + n_isl * 24 + side
    count_mean, compact_mean = statistics.fmean(count_ms), statistics.fmean(compact_ms)
    achieved = alg_compact / (compact_mean * 1e-3) / 1e9
    traffic = profiled_traffic("daq_compact_kernel", "full_fill")

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(elapsed_ms / K, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"full fill: {C} calorimeters x 54 crystals x 560,000 int16 samples "
                               f"({raw_bytes / 1e9:.4f} GB), literal noise sigma 3/crystal, T=30, pre=8, post=24, D=32",
                   "fills_per_step_per_gpu": 1, "raw_bytes_per_step_per_gpu": raw_bytes,
                   "l2": "inputs larger than L2 (1.45 GB per step vs 129 MB)", "parallelism": f"replicas x{ws}",
                   "tile": 448, "form": "two-pass: count kernel, scan, compact kernel"},
        "pct_of_hbm_peak": round(100.0 * value / ws / peak, 2),
        "pct_of_nominal_hbm": round(100.0 * value / ws / NOMINAL_HBM_GBS, 2),
        "latency_ms": {"p50": round(statistics.median(step_ms), 4),
                       "p99": round(float(np.percentile(step_ms, 99)), 4),
                       "max": round(max(step_ms), 4)},
        "kernels_ms": {"daq_prepare_kernel": round(statistics.fmean(prep_ms), 4),
                       "daq_count_kernel": round(count_mean, 4),
                       "daq_scan_kernel": round(statistics.fmean(scan_ms), 4),
                       "daq_compact_kernel": round(compact_mean, 4)},
        "count_kernel_gbs": round(alg_count / (count_mean * 1e-3) / 1e9, 1),
        "islands_per_fill": n_isl, "pool_rows_per_fill": n_rows,
        "coverage": round(n_rows / (C * N), 4),
        "output_over_input": round((n_rows * X * 2 + n_isl * 24) / raw_bytes, 4),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_kind,
                     "kernel": "daq_compact_kernel", "algorithmic_bytes_per_launch": alg_compact},
        "gpu_launches": 4 * K,
        "clocks": clocks.summary(),
    }

    # ---- end to end through the host-buffer entry point (before the sections that fill device memory)
    if not args.no_e2e:
        hdr_h = torch.empty(out.hdr_cap * 3, dtype=torch.int64).pin_memory()
        pool_h = torch.empty((rows_cap, X), dtype=torch.int16).pin_memory()
        counts_h = torch.zeros(4, dtype=torch.int64)
        io = daq.DaqHostIO(host.data_ptr(), samples.data_ptr(), hdr_h.data_ptr(), out.hdr_cap, pool_h.data_ptr(),
                           rows_cap, None, counts_h.data_ptr())
        pe, _ = make_p()
        pe.workspace, pe.workspace_bytes = workspace.data_ptr(), wsb
        Ke = max(3, min(K, args.e2e_steps))
        for _ in range(2):
            rc = daq.daq_process_fills_host(C, X, N, F, pe, isl, q.data_ptr(), io)
            assert rc == daq.DAQ_OK, rc
        # the link's rates just before the timed calls (others' traffic on a shared host lowers them)
        bw_before = copy_bandwidth(torch, dev, host, samples, pool_h, out.pool, int(counts_h[1]))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        call_ms = []
        e0.record(stream)
        for _ in range(Ke):
            tc = time.perf_counter()
            daq.daq_process_fills_host(C, X, N, F, pe, isl, q.data_ptr(), io)
            call_ms.append((time.perf_counter() - tc) * 1e3)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ems = e0.elapsed_time(e1)
        _, ems, e2e_value = replicas.aggregate(Ke * raw_bytes, ems, dev)
        d2h = 32 + int(counts_h[0]) * 24 + int(counts_h[1]) * X * 2
        bw = copy_bandwidth(torch, dev, host, samples, pool_h, out.pool, int(counts_h[1]))
        bw["before_e2e"] = {k: bw_before[k] for k in ("h2d_gbs", "d2h_gbs", "bidir_gbs", "median")}
        e2e_bound = raw_bytes / max(raw_bytes / bw["h2d_gbs"], d2h / bw["d2h_gbs"],
                                    (raw_bytes + d2h) / bw["bidir_gbs"]) if bw["h2d_gbs"] else None
        # the same through the packed host form (pool rows leave the GPU packed)
        pcap = daq.daq_pack_bound(rows_cap, X) + 64 * 8192
        pdev = torch.empty(pcap, dtype=torch.uint8, device=dev)
        phost = torch.empty(pcap, dtype=torch.uint8).pin_memory()
        pbytes = torch.zeros(1, dtype=torch.int64)
        pp_ = make_p()[0]
        pp_.workspace, pp_.workspace_bytes = workspace.data_ptr(), wsb
        pp_.flags |= daq.DAQ_PACK_POOL
        io.packed_dev, io.packed_dev_cap = pdev.data_ptr(), pcap
        io.packed_host, io.packed_host_cap, io.packed_bytes_host = phost.data_ptr(), pcap, pbytes.data_ptr()
        for _ in range(2):
            rc = daq.daq_process_fills_host(C, X, N, F, pp_, isl, q.data_ptr(), io)
            assert rc == daq.DAQ_OK, rc
        barrier()
        pk_call_ms = []
        e0.record(stream)
        for _ in range(Ke):
            tc = time.perf_counter()
            daq.daq_process_fills_host(C, X, N, F, pp_, isl, q.data_ptr(), io)
            pk_call_ms.append((time.perf_counter() - tc) * 1e3)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        _, pms, pk_value = replicas.aggregate(Ke * raw_bytes, e0.elapsed_time(e1), dev)
        pk_d2h = 32 + int(counts_h[0]) * 24 + int(pbytes.item())
        del pdev, phost
        result["e2e"] = {"value": round(e2e_value, 2), "unit": UNIT,
                         "h2d_bytes_per_step": raw_bytes, "d2h_bytes_per_step": d2h, "steps": Ke,
                         "ms_per_step": round(ems / Ke, 3),
                         "call_ms": {"min": round(min(call_ms), 3), "p50": round(statistics.median(call_ms), 3),
                                     "max": round(max(call_ms), 3), "all": [round(t, 2) for t in call_ms]},
                         "api": "daq_process_fills_host (pinned host buffers; copy-in, processing and copy-out "
                                "pipelined over calorimeter chunks)",
                         "copy_bandwidth": bw,
                         "bound_gbs": None if e2e_bound is None else round(e2e_bound, 2),
                         "packed": {"value": round(pk_value, 2), "unit": UNIT, "ms_per_step": round(pms / Ke, 3),
                                    "call_ms": {"min": round(min(pk_call_ms), 3),
                                                "p50": round(statistics.median(pk_call_ms), 3),
                                                "max": round(max(pk_call_ms), 3),
                                                "all": [round(t, 2) for t in pk_call_ms]},
                                    "h2d_bytes_per_step": raw_bytes, "d2h_bytes_per_step": pk_d2h,
                                    "api": "daq_process_fills_host with DAQ_PACK_POOL (pool rows packed losslessly "
                                           "on the GPU before the copy back)"}}

    # ---- batched form: 16 uneven fills in one tuned, graph-captured launch
    if not args.no_batched and not args.quick:
        result["batched"] = bench_batched(args, torch, dev, daq, synth, W)

    # ---- served form: request loop with admission, overlap and resident Q
    if not args.no_served and not args.quick:
        result["served"] = bench_served(args, torch, dev, daq, synth, W, samples)

    # ---- stress batch: 48 fills (69.67 GB) in one call, output sizes computed on the device
    if not args.no_stress and not args.quick:
        result["stress"] = bench_stress(args, torch, dev, daq, synth, W)

    # ---- sparse regime: islands cover ~8% of the fill
    if not args.no_sparse and not args.quick:
        result["sparse"] = bench_sparse(args, torch, dev, daq, synth, W)
        result["sparse"]["forms"] = bench_sparse_forms(args, torch, dev, daq, synth, W)

    # ---- lossless packing of the pool rows
    if not args.no_pack and not args.quick:
        result["pack"] = bench_pack(args, torch, dev, daq, out.pool, n_rows)

    # ---- per-crystal full-resolution fill sum
    if not args.no_crystal_sum and not args.quick:
        result["crystal_sum"] = bench_crystal_sum(args, torch, dev, daq, samples)

    # ---- island-finding efficiency across thresholds (Fig. 2)
    if not args.no_threshold_scan and not args.quick and rank == 0:
        scan = threshold_scan(torch, dev, daq, synth, W)
        result["threshold_scan"] = {"datasets": scan["datasets"],
                                    "slope": {t: v["slope"] for t, v in scan["thresholds"].items()},
                                    "corr": {t: v["corr"] for t, v in scan["thresholds"].items()},
                                    "ratio_of_totals": {t: v["ratio_of_totals"] for t, v in scan["thresholds"].items()}}

    # ---- single-pass plain kernel (grid -1): one CTA per tile, no persistence
    if not args.quick:
        pp, _ = make_p(grid=-1)
        pp.workspace, pp.workspace_bytes = workspace.data_ptr(), wsb
        Kp = max(3, min(K, 200))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(3):
                call(pp)
            e0.record(stream)
            for _ in range(Kp):
                call(pp)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        result["single_pass_kernel"] = {"value": round(Kp * raw_bytes / (e0.elapsed_time(e1) * 1e-3) / 1e9, 2),
                                        "unit": UNIT, "steps": Kp,
                                        "form": "single-pass plain kernel (grid -1), one CTA per tile"}

    # ---- CPU baseline: the oracle on a bounded sample of the same fill (rank 0)
    if rank == 0 and not args.no_cpu_baseline:
        gbs, dt, reps, threads, nbytes = run_cpu_oracle(host.numpy(), params, args.cpu_seconds)
        result["cpu_baseline"] = {"value": round(gbs, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                                  "sample": f"the whole 24-calorimeter fill ({nbytes} B) x {reps} passes, "
                                            f"{dt:.1f} s, calorimeter-fills spread over {threads} host threads"}
        # one thread on one calorimeter-fill (the oracle as a plain serial program)
        g1, dt1, reps1, _, nb1 = run_cpu_oracle(host.numpy(), params, min(3.0, args.cpu_seconds), calos=1, threads=1)
        result["cpu_baseline"]["single_thread"] = {
            "value": round(g1, 4), "unit": UNIT, "cores": 1,
            "sample": f"one calorimeter-fill ({nb1} B) x {reps1} passes, {dt1:.1f} s, one host thread"}
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return result if rank == 0 else None


def bench_batched(args, torch, dev, daq, synth, W, w=None, plain_flags=0) -> dict:
    """The batching workload: 16 fills x 24 calorimeters, lengths uniform in
    [80k, 560k] samples and pulse rates x log-uniform[0.2, 5], processed by
    one tuned plan replayed as a CUDA graph; Q accumulates over the fills.
    `w` replaces the workload (same shape); plain_flags are the plain form's
    processing flags (the tuned plan chooses its own)."""
    import numpy as np
    w = W.BATCH_UNEVEN if w is None else w
    params = w.params()
    fl, rate = w.plan()
    F, C, X, N = w.n_fills, w.n_calo, 54, w.n_samples
    cfg = w.config()
    samples = torch.empty((F, C, X, N), dtype=torch.int16, device=dev)
    stage = torch.empty((1, C, X, N), dtype=torch.int16).pin_memory()
    t0 = time.perf_counter()
    for f in range(F):
        synth.generate(cfg, fill_len=fl, rate=rate, out=stage.numpy(), n_threads=os.cpu_count() or 1,
                       fills=(f, 1))
        samples[f].copy_(stage[0], non_blocking=False)
    gen_s = time.perf_counter() - t0
    del stage
    raw = int(C * X * 2 * int(np.asarray(fl, np.int64).sum()))
    rows = C * int(np.asarray(fl, np.int64).sum())
    out = daq.Outputs(torch, dev, F, C, X, rows // 4 + F * C + 1, rows)
    q = torch.zeros(daq.q_size(C, N, params["decim"]), dtype=torch.int64, device=dev)
    fl_d = torch.as_tensor(np.asarray(fl, np.int32), device=dev)
    t1 = time.perf_counter()
    # tuned on this batch's own data (the library remembers a choice per shape and parameters, and
    # the dense and sparse batches share both)
    plan = daq.BatchPlan(samples, q, out, fill_len=fl_d, tune=True, force=True, **params)
    tune_s = time.perf_counter() - t1
    tuning = plan.tuning()
    stream = torch.cuda.Stream(dev)
    for _ in range(3):
        plan.launch(stream)
    torch.cuda.synchronize(dev)
    counts = out.counts.cpu().numpy()
    status = daq.daq_status_from_counts(counts)
    if status != daq.DAQ_OK:
        raise daq.DaqError(status, "batched warm-up")
    Kb = max(3, min(args.steps, args.batched_steps))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(Kb)]
    for k in range(Kb):
        evs[k][0].record(stream)
        plan.launch(stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = evs[0][0].elapsed_time(evs[-1][1])
    plan.close()
    # the plain form on the same fills: the default kernels (two-pass, library
    # tile), one daq_process_fills call per fill, no graph and no tuning; each
    # call writes its fill's records and rows from the start of the outputs
    pp = daq.make_params(**params, stream=stream, flags=plain_flags)
    wsb1 = daq.daq_workspace_size(C, X, N, 1, pp)
    ws1 = torch.empty(wsb1, dtype=torch.uint8, device=dev)
    pp.workspace, pp.workspace_bytes = ws1.data_ptr(), wsb1
    isl = out.struct()
    fill_bytes = C * X * N * 2

    def plain_batch():
        for f in range(F):
            pp.fill_len = fl_d.data_ptr() + 4 * f
            pp.fill_base = f
            rc = daq.daq_process_fills(samples.data_ptr() + f * fill_bytes, C, X, N, 1, pp, isl, q.data_ptr())
            if rc != daq.DAQ_OK:
                raise daq.DaqError(rc, "plain form")

    for _ in range(2):
        plain_batch()
    torch.cuda.synchronize(dev)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(Kb):
        plain_batch()
    p1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = p0.elapsed_time(p1)
    plain = {"value": round(Kb * raw / (plain_ms * 1e-3) / 1e9, 2), "unit": UNIT, "steps": Kb,
             "ms_per_batch": round(plain_ms / Kb, 4),
             "form": "default two-pass kernels, one daq_process_fills call per fill (16 calls per batch), "
                     "no graph, no tuning" + (f", flags {plain_flags}" if plain_flags else "")}
    del ws1
    res = {"value": round(Kb * raw / (total_ms * 1e-3) / 1e9, 2), "unit": UNIT, "steps": Kb,
           "ms_per_batch": round(total_ms / Kb, 4),
           "latency_ms": {"p50": round(statistics.median(ms), 4), "p99": round(float(np.percentile(ms, 99)), 4)},
           "pct_of_hbm_peak": round(100.0 * Kb * raw / (total_ms * 1e-3) / 1e9 / measured_peaks()[0], 2),
           "workload": "16 fills x 24 calorimeters x 54 crystals, lengths uniform in [80k, 560k] samples "
                       "(pitch 560,000), pulse rate x log-uniform[0.2, 5] per fill, T=30, pre=8, post=24, D=32"
                       + ("" if w is W.BATCH_UNEVEN else f"; {w.name}"),
           "raw_bytes_per_batch": raw, "islands_per_batch": int(counts[0]), "pool_rows_per_batch": int(counts[1]),
           "coverage": round(int(counts[1]) / rows, 4),
           "launch": "one CUDA graph launch per batch (daq_batch_plan_create / daq_batch_launch)",
           "tuned": {"tile": tuning["tile"], "grid": tuning["grid"], "flags": tuning.get("flags", 0),
                     "candidates": tuning["n_tried"],
                     "ms": round(tuning["ms"], 4), "ms_default_config": round(tuning["ms_default"], 4),
                     "tuning_s": round(tune_s, 2)},
           "gpu_launches": 4 * Kb, "generation_s": round(gen_s, 1),
           "plain_form": plain, "batched_over_plain": round((Kb * raw / (total_ms * 1e-3)) / (Kb * raw / (plain_ms * 1e-3)), 4)}
    del samples, out, q
    torch.cuda.empty_cache()
    return res


def copy_bandwidth(torch, dev, host_in, dev_in, host_out, dev_out, out_rows: int, reps: int = 3) -> dict:
    """Pinned host<->device copy rates of this machine (the bound of the end-to-end
    form): the input host->device, the pool rows device->host, and both at once
    on two streams.  Plain cudaMemcpyAsync through torch."""
    a, b = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    src_h, dst_d = host_in.view(-1), dev_in.view(-1)
    n_out = max(1, out_rows) * dev_out.shape[1]
    src_d, dst_h = dev_out.view(-1)[:n_out], host_out.view(-1)[:n_out]
    nb_in, nb_out = src_h.numel() * 2, n_out * 2

    def timed(fn):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(reps):
            e0.record(torch.cuda.current_stream(dev))
            fn()
            for st in (a, b):
                torch.cuda.current_stream(dev).wait_stream(st)
            e1.record(torch.cuda.current_stream(dev))
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
        return min(times), statistics.median(times)

    def h2d():
        a.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(a):
            dst_d.copy_(src_h, non_blocking=True)

    def d2h():
        b.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(b):
            dst_h.copy_(src_d, non_blocking=True)

    def both():
        h2d()
        d2h()

    (t_in, m_in), (t_out, m_out), (t_both, m_both) = timed(h2d), timed(d2h), timed(both)
    gbs = lambda nb, ms: round(nb / (ms * 1e-3) / 1e9, 1)
    return {"h2d_gbs": gbs(nb_in, t_in), "d2h_gbs": gbs(nb_out, t_out), "bidir_gbs": gbs(nb_in + nb_out, t_both),
            "median": {"h2d_gbs": gbs(nb_in, m_in), "d2h_gbs": gbs(nb_out, m_out),
                       "bidir_gbs": gbs(nb_in + nb_out, m_both)},
            "method": f"best (and median) of {reps} pinned cudaMemcpyAsync of the fill (h2d) and of its pool rows "
                      "(d2h), alone and concurrently on two streams"}


def time_calls(torch, dev, daq, x, F, C, X, N, params, K: int, out=None, warm: int = 2):
    """Run daq_process_fills K times on device samples x[F][C][X][N].  Returns
    (total ms of the K calls, per-step ms list and kernel means from a second
    run with per-kernel events, counts)."""
    stream = torch.cuda.Stream(dev)
    if out is None:
        out = daq.Outputs(torch, dev, F, C, X, F * C * N // 2 + F * C + 1, F * C * N)
    q = torch.zeros(max(1, daq.q_size(C, N, params["decim"])), dtype=torch.int64, device=dev)
    p = daq.make_params(**params, stream=stream)
    wsb = daq.daq_workspace_size(C, X, N, F, p)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    p.workspace, p.workspace_bytes = ws.data_ptr(), wsb
    isl = out.struct()
    for _ in range(warm):
        rc = daq.daq_process_fills(x.data_ptr(), C, X, N, F, p, isl, q.data_ptr())
        assert rc == daq.DAQ_OK, rc
    # the total from two bracketing events; per-step and per-kernel times from a
    # second run with events between the kernels
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    t0.record(stream)
    for _ in range(K):
        daq.daq_process_fills(x.data_ptr(), C, X, N, F, p, isl, q.data_ptr())
    t1.record(stream)
    torch.cuda.synchronize(dev)
    total = t0.elapsed_time(t1)
    Kd = max(3, min(K, 200))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(Kd)]
    for row in evs:
        for e in row:
            e.record(stream)
    arrs = [(ctypes.c_void_p * 5)(*[e.cuda_event for e in row]) for row in evs]
    torch.cuda.synchronize(dev)
    for k in range(Kd):
        p.events = ctypes.cast(arrs[k], ctypes.c_void_p).value
        daq.daq_process_fills(x.data_ptr(), C, X, N, F, p, isl, q.data_ptr())
    p.events = None
    torch.cuda.synchronize(dev)
    ms = [r[0].elapsed_time(r[4]) for r in evs]
    kern = {name: round(statistics.fmean(r[i].elapsed_time(r[i + 1]) for r in evs), 4)
            for i, name in enumerate(["daq_prepare_kernel", "daq_count_kernel", "daq_scan_kernel",
                                      "daq_compact_kernel"])}
    counts = out.counts.cpu().numpy()
    del ws, q
    return total, ms, kern, counts


def bench_sparse(args, torch, dev, daq, synth, W) -> dict:
    """The sparse regime: per-crystal noise 3/sqrt(54), so the 54-crystal sum
    has sigma ~3 ADC and islands cover a small part of the fill (the data
    reduction the experiment's DAQ is built for)."""
    import numpy as np
    w = W.SPARSE_FULL_FILL
    params = w.params()
    F, C, X, N = 1, w.n_calo, 54, w.n_samples
    stage = torch.empty((1, C, X, N), dtype=torch.int16).pin_memory()
    synth.generate(w.config(), out=stage.numpy(), n_threads=os.cpu_count() or 1)
    x = stage.to(dev)
    del stage
    K = max(3, min(args.steps, args.sparse_steps))
    # DAQ_SPARSE: the compact pass takes only the tiles that hold a marked sample
    total, ms, kern, counts = time_calls(torch, dev, daq, x, F, C, X, N, dict(params, flags=daq.DAQ_SPARSE), K)
    total_d, _, kern_d, _ = time_calls(torch, dev, daq, x, F, C, X, N, params, K)
    raw = F * C * X * N * 2
    value = K * raw / (total * 1e-3) / 1e9
    peak = measured_peaks()[0]
    cov = int(counts[1]) / (F * C * N)
    out_bytes = int(counts[1]) * X * 2 + int(counts[0]) * 24
    ceiling = peak / (2 + out_bytes / raw)     # two full passes over the input plus the output writes
    once = peak / (1 + out_bytes / raw)        # the input read once plus the output writes
    del x
    torch.cuda.empty_cache()
    return {"value": round(value, 2), "unit": UNIT, "steps": K, "ms_per_step": round(total / K, 4),
            "latency_ms_p99": round(float(np.percentile(ms, 99)), 4),
            "workload": "full fill 24 x 54 x 560,000 int16, per-crystal noise sigma 3/sqrt(54) (sum sigma ~3 ADC), "
                        "T=30, pre=8, post=24, D=32",
            "flags": "DAQ_SPARSE (the compact pass takes only tiles that hold a marked sample)",
            "coverage": round(cov, 4), "islands_per_fill": int(counts[0]), "output_bytes_per_fill": out_bytes,
            "output_over_input": round(out_bytes / raw, 4), "data_reduction": round(raw / max(1, out_bytes), 1),
            "pct_of_hbm_peak": round(100.0 * value / peak, 2),
            "two_pass_ceiling_gbs": round(ceiling, 1), "frac_of_two_pass_ceiling": round(value / ceiling, 4),
            "read_once_ceiling_gbs": round(once, 1), "frac_of_read_once_ceiling": round(value / once, 4),
            "kernels_ms": kern, "gpu_launches": 4 * K,
            "default_flags": {"value": round(K * raw / (total_d * 1e-3) / 1e9, 2), "ms_per_step": round(total_d / K, 4),
                              "kernels_ms": kern_d}}


def plan_tile(daq, F, C, X, N, params) -> int | None:
    """The tile width the default plan takes for these sizes and windows (read
    back through its tile count)."""
    tiles = daq.daq_trace_tiles(C, X, N, F, daq.make_params(**params))
    for tw in (448, 384, 224, 128):
        if tiles == F * C * -(-N // tw):
            return tw
    return None


def bench_stress(args, torch, dev, daq, synth, W) -> dict:
    """The stress workload: 48 fills x 24 calorimeters x 54 x 560,000 int16
    (69.67 GB device-resident), 10x pulse rate, T=15, post=64, D in {8, 32},
    one call over all 48 fills; the fills cycle over 4 distinct generated
    fills (the kernels cannot tell)."""
    import numpy as np
    w = W.STRESS if args.stress_fills == W.STRESS.n_fills else W.scaled(W.STRESS, n_fills=args.stress_fills)
    params = w.params()
    F, C, X, N = w.n_fills, w.n_calo, 54, w.n_samples
    free, _ = torch.cuda.mem_get_info(dev)
    need = 2 * F * C * X * N * 2 + (8 << 30)
    if free < need:
        return {"skipped": f"needs {need / 1e9:.0f} GB free device memory, {free / 1e9:.0f} GB free"}
    n_distinct = min(4, F)
    t0 = time.perf_counter()
    x = torch.empty((F, C, X, N), dtype=torch.int16, device=dev)
    stage = torch.empty((1, C, X, N), dtype=torch.int16).pin_memory()
    for d in range(n_distinct):
        synth.generate(w.config(), out=stage.numpy(), n_threads=os.cpu_count() or 1, fills=(d, 1))
        x[d].copy_(stage[0])
    for f in range(n_distinct, F):
        x[f].copy_(x[f % n_distinct])
    del stage
    gen_s = time.perf_counter() - t0
    raw = F * C * X * N * 2
    out = daq.Outputs(torch, dev, F, C, X, F * C * 1024, F * C * N)
    Ks = max(3, min(args.steps, args.stress_steps))
    total, ms, kern, counts = time_calls(torch, dev, daq, x, F, C, X, N, params, Ks, out=out)
    status = daq.daq_status_from_counts(counts)
    res = {"value": round(Ks * raw / (total * 1e-3) / 1e9, 2), "unit": UNIT, "steps": Ks,
           "ms_per_batch": round(total / Ks, 3), "latency_ms_p99": round(float(np.percentile(ms, 99)), 3),
           "pct_of_hbm_peak": round(100.0 * Ks * raw / (total * 1e-3) / 1e9 / measured_peaks()[0], 2),
           "workload": f"{F} fills x 24 calorimeters x 54 crystals x 560,000 int16 ({raw / 1e9:.2f} GB device-resident), "
                       "10x pulse rate (~15,000 pulses per calorimeter-fill), T=15, pre=8, post=64, D=8 and 32; "
                       "fills cycle over 4 distinct generated fills",
           "raw_bytes_per_batch": raw, "islands_per_batch": int(counts[0]), "pool_rows_per_batch": int(counts[1]),
           "coverage": round(int(counts[1]) / (F * C * N), 6), "status": status,
           "output_sizes": "computed on the device (counts) in the same call", "gpu_launches": 4 * Ks,
           "kernels_ms": kern, "tile": plan_tile(daq, F, C, X, N, params),
           "generation_s": round(gen_s, 1)}
    del x, out
    torch.cuda.empty_cache()
    return res


def bench_crystal_sum(args, torch, dev, daq, samples) -> dict:
    """Per-crystal full-resolution fill sum on the full fill: int64 Q of
    24 x 54 x 560,000 bins resident on the device, one call per fill."""
    F, C, X, N = (int(v) for v in samples.shape)
    q = torch.zeros((C, X, N), dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream(dev)
    p = daq.make_params(stream=stream)
    need = daq.daq_crystal_sum_workspace_size(C, X, F)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    p.workspace, p.workspace_bytes = ws.data_ptr(), need
    for _ in range(3):
        assert daq.daq_crystal_sum(samples.data_ptr(), C, X, N, F, p, q.data_ptr()) == daq.DAQ_OK
    K = max(3, min(args.steps, args.crystal_steps))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(K):
        daq.daq_crystal_sum(samples.data_ptr(), C, X, N, F, p, q.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / K
    raw = F * C * X * N * 2
    alg = raw + C * X * N * 16
    peak = measured_peaks()[0]
    del q, ws
    torch.cuda.empty_cache()
    return {"value": round(raw / (ms * 1e-3) / 1e9, 2), "unit": UNIT, "steps": K, "ms_per_fill": round(ms, 4),
            "workload": "full fill 24 x 54 x 560,000 int16 into int64 Q[24][54][560,000] (5.8 GB, device-resident)",
            "roofline": {"bound": "hbm", "achieved": round(alg / (ms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4),
                         "algorithmic_bytes_per_launch": alg,
                         "note": "2 B per sample read + 16 B per crystal-sample of Q read and written"},
            "gpu_launches": 2 * K}


def bench_pack(args, torch, dev, daq, pool, rows: int) -> dict:
    """Lossless packing of the full fill's pool rows (what leaves the GPU)."""
    X = int(pool.shape[1])
    cap = daq.daq_pack_bound(rows, X)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    need = daq.daq_pack_workspace_size(rows, X)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream(dev)

    def call():
        rc = daq.daq_pack_pool(pool.data_ptr(), rows, X, out.data_ptr(), cap, nbytes.data_ptr(), ws.data_ptr(),
                               need, stream.cuda_stream)
        assert rc == daq.DAQ_OK, rc

    for _ in range(3):
        call()
    K = max(3, min(args.steps, args.pack_steps))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(K):
        call()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / K
    n = int(nbytes.item())
    raw = rows * X * 2
    alg = 2 * raw + n        # the pool is read by the size pass and by the write pass
    peak = measured_peaks()[0]
    # decoding the stream back into pool rows (checked against the pool once)
    back = torch.empty((rows, X), dtype=torch.int16, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)

    def decode():
        rc = daq.daq_unpack_pool(out.data_ptr(), n, rows, X, back.data_ptr(), err.data_ptr(), stream.cuda_stream)
        assert rc == daq.DAQ_OK, rc

    decode()
    torch.cuda.synchronize(dev)
    assert int(err.item()) == 0 and torch.equal(back, pool[:rows]), "decoded pool differs"
    e0.record(stream)
    for _ in range(K):
        decode()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ums = e0.elapsed_time(e1) / K
    del out, ws, back
    torch.cuda.empty_cache()
    return {"value": round(raw / (ms * 1e-3) / 1e9, 2), "unit": "GB/s of pool rows packed", "steps": K,
            "ms_per_fill": round(ms, 4), "pool_bytes": raw, "packed_bytes": n,
            "compression_ratio": round(raw / max(1, n), 3),
            "workload": "pool rows of the full fill (24 x 54 x 560,000, T=30, pre=8, post=24)",
            "roofline": {"bound": "hbm", "achieved": round(alg / (ms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4), "algorithmic_bytes_per_launch": alg},
            "unpack": {"value": round(raw / (ums * 1e-3) / 1e9, 2), "unit": "GB/s of pool rows decoded",
                       "ms_per_fill": round(ums, 4), "steps": K, "gpu_launches": K},
            "gpu_launches": 5 * K}


THRESHOLDS = (5, 10, 15, 20, 30, 50, 100, 300, 1000)


def threshold_scan(torch, dev, daq, synth, W, n_fills: int = 12, n_calo: int = 2, thresholds=THRESHOLDS) -> dict:
    """Island-finding efficiency across thresholds (Fig. 2): datasets are
    calorimeter-fills of the sparse regime with pulse rates x
    log-uniform[0.2, 5]; the islands the CUDA path identifies in each are
    compared with the truth islands of its injected pulse list (each pulse's
    samples above T, widened by the windows and merged;
    paper_1611_04959_gb300.fig2)."""
    from paper_1611_04959_gb300 import fig2
    w = W.scaled(W.SPARSE_FULL_FILL, n_fills=n_fills, n_calo=n_calo)
    N = w.n_samples
    _, rates = synth.fill_plan(w.synth["seed"] + 29, n_fills, N, N, 0.2, 5.0)
    x = torch.from_numpy(synth.generate(w.config(), rate=rates, n_threads=os.cpu_count() or 1)).to(dev)
    truth = [[synth.pulses(w.config(), f, c, N, float(rates[f])) for c in range(n_calo)] for f in range(n_fills)]
    base = w.params()
    scan = fig2.threshold_scan(x, truth, base, thresholds)
    del x
    torch.cuda.empty_cache()
    return {"datasets": f"{n_fills * n_calo} calorimeter-fills (sparse regime: sum noise sigma ~3 ADC; pulse rate x "
                        "log-uniform[0.2, 5] per fill); truth = islands of the injected pulse list at the same "
                        "threshold and windows",
            "pre": base["pre"], "post": base["post"],
            "injected_pulses": [len(truth[f][c]) for f in range(n_fills) for c in range(n_calo)],
            "thresholds": scan["thresholds"]}


def burst_schedule(n_fills: int, speed: float, t0_us: float) -> list:
    """Arrival times (us) of the accelerator cycle replayed `speed` times
    faster: bursts of 8 fills 10 ms apart, two bursts per 1.4 s cycle (the
    second half a cycle after the first)."""
    cycle, spacing = 1.4e6 / speed, 10e3 / speed
    out = []
    for i in range(n_fills):
        c, b, k = i // 16, (i // 8) % 2, i % 8
        out.append(t0_us + c * cycle + b * cycle / 2 + k * spacing)
    return out


def bench_served(args, torch, dev, daq, synth, W, samples0) -> dict:
    """The serving workload: a stream of 24-calorimeter fills arriving in the
    accelerator's burst pattern at 1x, 10x and 100x, served by the request
    loop (40 GB slot budget, 4 streams, Q resident across every fill) from a
    pool of device-resident fills; plus a saturated run (all fills at once)."""
    import numpy as np
    w = W.SERVING
    params = w.params()
    C, X, N = w.n_calo, 54, w.n_samples
    n_pool = max(1, args.serve_pool)
    cfg = W.scaled(w, n_fills=n_pool).config()
    pool = [samples0[0]]
    stage = torch.empty((1, C, X, N), dtype=torch.int16).pin_memory()
    for f in range(1, n_pool):
        synth.generate(cfg, out=stage.numpy(), n_threads=os.cpu_count() or 1, fills=(f, 1))
        pool.append(stage[0].to(dev))
    del stage
    # host input first: measured after the device-resident runs below, its 1x
    # latencies came out several times longer than on a fresh server process
    host_rates = served_host_input(args, torch, dev, daq, params, C, X, N, pool[: min(2, n_pool)])
    budget = 40 << 30
    srv = daq.DaqServer(C, X, N, budget, **params, n_streams=4, auto_release=True, device=dev)
    st0 = srv.stats()
    # warm-up
    for k in range(4):
        srv.submit(pool[k % n_pool])
    srv.drain(120.0)
    srv.records(clear=True)
    rates = {}
    for speed, n in ((1, args.serve_fills_1x), (10, args.serve_fills), (100, args.serve_fills)):
        t0 = srv.now_us() + 50e3
        arr = burst_schedule(n, speed, t0)
        with ClockSampler(dev.index or 0) as clk:
            for i, a in enumerate(arr):
                srv.submit(pool[i % n_pool], arrival_us=a)
            srv.drain(600.0)
        recs = srv.records(clear=True)
        sm = daq.daq_serving_summarize(recs)
        lat = [r.t_done - r.t_arrival for r in recs]
        offered = n * C * X * N * 2 / ((arr[-1] - arr[0]) * 1e-6) / 1e9 if n > 1 else None
        rates[f"{speed}x"] = {"fills": n, "fill_spacing_ms": 10.0 / speed, "cycle_ms": 1400.0 / speed,
                              "latency_ms": {"p50": round(sm.latency_p50_us / 1e3, 4),
                                             "p99": round(sm.latency_p99_us / 1e3, 4),
                                             "max": round(sm.latency_max_us / 1e3, 4)},
                              "p99_under_fill_spacing": bool(sm.latency_p99_us < 10e3 / speed),
                              "deadtime": round(sm.deadtime, 4),
                              "served_gbs": round(sm.gbs, 2),
                              "offered_gbs": None if offered is None else round(offered, 2),
                              "clocks": clk.summary()}
        assert all(r.status == 0 for r in recs), "served fill failed"
        del lat
    # saturated: every fill arrives at once; throughput of the overlapped stream
    n_sat = args.serve_fills_saturated
    for i in range(n_sat):
        srv.submit(pool[i % n_pool])
    srv.drain(600.0)
    recs = srv.records(clear=True)
    sm = daq.daq_serving_summarize(recs)
    busy = max(r.t_done for r in recs) - min(r.t_start for r in recs)
    sat_gbs = n_sat * C * X * N * 2 / (busy * 1e-6) / 1e9
    st = srv.stats()
    srv.close()
    return {"workload": "stream of 24 x 54 x 560,000 int16 fills (1.4515 GB each) from a pool of "
                        f"{n_pool} device-resident generated fills; bursts of 8 fills 10 ms apart, 2 bursts per "
                        "1.4 s cycle, replayed at 1x / 10x / 100x; T=30, pre=8, post=24, D=32",
            "budget_bytes": budget, "slots": st0["n_slots"], "slot_bytes": st0["slot_bytes"],
            "streams": st0["n_streams"], "rates": rates,
            "saturated": {"value": round(sat_gbs, 2), "unit": UNIT, "fills": n_sat,
                          "pct_of_hbm_peak": round(100.0 * sat_gbs / measured_peaks()[0], 2),
                          "max_running": st["max_running"],
                          "latency_ms_p50": round(sm.latency_p50_us / 1e3, 3)},
            "q": "one int64 Q histogram resident on the device across every served fill",
            "host_input": host_rates}


def bench_sparse_forms(args, torch, dev, daq, synth, W) -> dict:
    """The batched and served forms in the sparse regime (per-crystal noise
    3/sqrt(54): islands on a few percent of the samples): the batching
    workload's 16 uneven fills with that noise under a tuned plan, and a served
    stream of sparse fills with DAQ_SPARSE at 10x and saturated."""
    import math
    import numpy as np
    sig = 3.0 / math.sqrt(54.0)
    import dataclasses
    wb = dataclasses.replace(W.scaled(W.BATCH_UNEVEN, noise_sigma=sig), name="per-crystal noise sigma 3/sqrt(54)")
    out = {"batched": bench_batched(args, torch, dev, daq, synth, W, w=wb, plain_flags=daq.DAQ_SPARSE)}
    torch.cuda.empty_cache()
    w = W.SPARSE_FULL_FILL
    params = w.params()
    C, X, N = w.n_calo, 54, w.n_samples
    n_pool = max(1, args.serve_pool)
    cfg = W.scaled(w, n_fills=n_pool).config()
    pool = []
    stage = torch.empty((1, C, X, N), dtype=torch.int16).pin_memory()
    for f in range(n_pool):
        synth.generate(cfg, out=stage.numpy(), n_threads=os.cpu_count() or 1, fills=(f, 1))
        pool.append(stage[0].to(dev))
    del stage
    srv = daq.DaqServer(C, X, N, 40 << 30, **params, n_streams=4, auto_release=True, device=dev,
                        flags=daq.DAQ_SPARSE)
    for k in range(4):
        srv.submit(pool[k % n_pool])
    srv.drain(120.0)
    srv.records(clear=True)
    n = args.serve_fills
    t0 = srv.now_us() + 50e3
    arr = burst_schedule(n, 10, t0)
    with ClockSampler(dev.index or 0) as clk:
        for i, a in enumerate(arr):
            srv.submit(pool[i % n_pool], arrival_us=a)
        srv.drain(600.0)
    recs = srv.records(clear=True)
    assert all(r.status == 0 for r in recs), "served sparse fill failed"
    sm = daq.daq_serving_summarize(recs)
    n_sat = args.serve_fills_saturated
    for i in range(n_sat):
        srv.submit(pool[i % n_pool])
    srv.drain(600.0)
    recs_s = srv.records(clear=True)
    assert all(r.status == 0 for r in recs_s), "served sparse fill failed"
    busy = max(r.t_done for r in recs_s) - min(r.t_start for r in recs_s)
    sat = n_sat * C * X * N * 2 / (busy * 1e-6) / 1e9
    st = srv.stats()
    srv.close()
    del pool
    torch.cuda.empty_cache()
    peak = measured_peaks()[0]
    out["served"] = {"workload": f"stream of sparse 24 x 54 x 560,000 fills (per-crystal noise sigma 3/sqrt(54)) from "
                                 f"{n_pool} device-resident fills, DAQ_SPARSE; bursts of 8 fills 1 ms apart (10x)",
                     "10x": {"fills": n, "latency_ms": {"p50": round(sm.latency_p50_us / 1e3, 4),
                                                        "p99": round(sm.latency_p99_us / 1e3, 4)},
                             "p99_under_fill_spacing": bool(sm.latency_p99_us < 1e3), "deadtime": round(sm.deadtime, 4),
                             "served_gbs": round(sm.gbs, 2), "clocks": clk.summary()},
                     "saturated": {"value": round(sat, 2), "unit": UNIT, "fills": n_sat,
                                   "pct_of_hbm_peak": round(100.0 * sat / peak, 2), "max_running": st["max_running"]}}
    out["batched"]["pct_of_hbm_peak"] = round(100.0 * out["batched"]["value"] / peak, 2)
    return out


def served_host_input(args, torch, dev, daq, params, C, X, N, dev_fills) -> dict:
    """The served workload with every fill coming from page-locked host memory:
    the server copies each fill into its slot (host-to-device) before processing
    it, so a fill's latency includes the copy.  1x and 10x burst schedules; the
    link's measured host-to-device rate is the bound."""
    import numpy as np
    hosts = []
    for f in dev_fills:
        h = torch.empty((C, X, N), dtype=torch.int16).pin_memory()
        h.copy_(f)
        hosts.append(h)
    fill_bytes = C * X * N * 2
    # the link's host-to-device rate, one fill copied at a time
    dtmp = torch.empty((C, X, N), dtype=torch.int16, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dtmp.copy_(hosts[0], non_blocking=True)
    e0.record()
    for _ in range(4):
        dtmp.copy_(hosts[0], non_blocking=True)
    e1.record()
    torch.cuda.synchronize(dev)
    h2d_gbs = 4 * fill_bytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del dtmp
    srv = daq.DaqServer(C, X, N, 40 << 30, **params, n_streams=4, host_input=True, auto_release=True, device=dev)
    for k in range(4):
        srv.submit(hosts[k % len(hosts)])
    srv.drain(120.0)
    srv.records(clear=True)
    out = {"h2d_gbs_measured": round(h2d_gbs, 2), "copy_ms_per_fill_at_link_rate": round(fill_bytes / h2d_gbs / 1e6, 3)}
    for speed, n in ((1, args.serve_fills_1x), (10, args.serve_fills_host_10x)):
        t0 = srv.now_us() + 50e3
        arr = burst_schedule(n, speed, t0)
        with ClockSampler(dev.index or 0) as clk:
            for i, a in enumerate(arr):
                srv.submit(hosts[i % len(hosts)], arrival_us=a)
            srv.drain(600.0)
        recs = srv.records(clear=True)
        assert all(r.status == 0 for r in recs), "served host-input fill failed"
        sm = daq.daq_serving_summarize(recs)
        offered = n * fill_bytes / ((arr[-1] - arr[0]) * 1e-6) / 1e9 if n > 1 else None
        out[f"{speed}x"] = {"fills": n, "fill_spacing_ms": 10.0 / speed,
                            "latency_ms": {"p50": round(sm.latency_p50_us / 1e3, 4),
                                           "p99": round(sm.latency_p99_us / 1e3, 4),
                                           "max": round(sm.latency_max_us / 1e3, 4)},
                            "p99_under_fill_spacing": bool(sm.latency_p99_us < 10e3 / speed),
                            "deadtime": round(sm.deadtime, 4), "served_gbs": round(sm.gbs, 2),
                            "offered_gbs": None if offered is None else round(offered, 2),
                            "clocks": clk.summary()}
    srv.close()
    del hosts
    return out


# ----------------------------------------------------------------------------- reference arm (oracle)
def bench_reference(args, ws, rank, local):
    if rank != 0:
        return None
    import numpy as np
    import oracle
    import synth
    from synth import workloads as W
    oracle.build()
    w = W.PLAIN_FULL_FILL
    params = w.params()
    threads = os.cpu_count() or 1
    calos = min(w.n_calo, threads)
    cfg = W.scaled(w, n_calo=calos).config()
    s = synth.generate(cfg, n_threads=threads)
    # bounded sample per step: `calos` calorimeters x `length` samples, sized so
    # that warm-up + timed steps end within about two minutes
    budget = max(0.05, min(2.0, 120.0 / max(1, args.steps + args.warmup)))
    t0 = time.perf_counter()
    oracle.process_fills(np.ascontiguousarray(s[:, :, :, :56_000]), params, n_threads=threads)
    per_sample = (time.perf_counter() - t0) / 56_000
    length = int(min(w.n_samples, max(4_000, budget / max(per_sample, 1e-12))) // 8 * 8)
    sub = np.ascontiguousarray(s[:, :, :, :length])
    for _ in range(args.warmup):
        oracle.process_fills(sub, params, n_threads=threads)
    times = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        oracle.process_fills(sub, params, n_threads=threads)
        times.append(time.perf_counter() - t1)
    total = sum(times)
    value = len(times) * sub.nbytes / total / 1e9
    sample = f"{calos} calorimeters x 54 crystals x first {length} samples of the fill per step ({sub.nbytes} B)"
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / len(times), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "full fill: 24 calorimeters x 54 crystals x 560,000 int16 samples (1.4515 GB), "
                               "literal noise sigma 3/crystal, T=30, pre=8, post=24, D=32",
                   "sample_per_step": sample},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="main measurement only (no plain or batched form)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 16-fill batched form")
    ap.add_argument("--batched-steps", type=int, default=30)
    ap.add_argument("--no-served", action="store_true", help="skip the served (request loop) form")
    ap.add_argument("--no-stress", action="store_true", help="skip the 48-fill (69.67 GB) stress batch")
    ap.add_argument("--stress-steps", type=int, default=10)
    ap.add_argument("--stress-fills", type=int, default=48, help="fills of the stress batch (48; fewer for profiling)")
    ap.add_argument("--no-sparse", action="store_true", help="skip the sparse-regime fill")
    ap.add_argument("--no-threshold-scan", action="store_true", help="skip the island-efficiency threshold scan")
    ap.add_argument("--no-crystal-sum", action="store_true", help="skip the per-crystal full-resolution fill sum")
    ap.add_argument("--crystal-steps", type=int, default=50)
    ap.add_argument("--no-pack", action="store_true", help="skip the pool-packing measurement")
    ap.add_argument("--pack-steps", type=int, default=50)
    ap.add_argument("--sparse-steps", type=int, default=1000)
    ap.add_argument("--serve-pool", type=int, default=4, help="distinct device fills the served stream cycles over")
    ap.add_argument("--serve-fills", type=int, default=1024, help="fills per served run at 10x and 100x")
    ap.add_argument("--serve-fills-1x", type=int, default=32, help="fills of the 1x run (1.4 s per 16 fills)")
    ap.add_argument("--serve-fills-saturated", type=int, default=256)
    ap.add_argument("--serve-fills-host-10x", type=int, default=64, help="fills of the host-input 10x run")
    ap.add_argument("--calos", type=int, default=24, help="calorimeters per fill (24; fewer only for profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        res = bench_reference(args, ws, rank, local)
    else:
        res = bench_gb300(args, ws, rank, local)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
