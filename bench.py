#!/usr/bin/env python
"""Particle-steps/s of the per-frame SIR tracker step on GB300 (one JSON line on rank 0).

Workload (single tracker at scale): a 512x512 synthetic video of 100 frames, a disk of
radius 5 moving (+1, -2) px/frame with noise sigma 5, tracked by 2^20 particles (random
walk sigma 1 px, init at the true start, Philox seed 1).  One bench step = the whole
100-frame track through the C ABI (pf_reset + 100 x pf_step_frame), frames resident in
HBM; L2 is flushed (a 512 MiB write) between timed steps, outside the timed events.
The headline arithmetic is FP16 (half2 propagation and likelihood, FP32 weights / scan);
REF64, F32 and BF16 are timed beside it on the same Philox stream, with their track
RMSE against the REF64 GPU track.

--impl reference times the CPU FP64 oracle (oracle/) on the host cores instead, each
step a bounded sample of the same workload (its first frames at full N).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W_, H_, T_, R_, N_, NOISE_, SEED_ = 512, 512, 100, 5, 1 << 20, 5.0, 1
WORKLOAD = ("single tracker at scale: 512x512 uint8 synthetic video, 100 frames, disk r=5 "
            "moving (+1,-2) px/frame, noise sigma 5, 2^20 particles, random walk sigma 1 px, Philox seed 1")
WORKLOAD_SHORT = "512x512 video, 100 frames, disk r=5 moving (+1,-2), noise 5, 2^20 particles, sigma 1 px, seed 1"
METRIC = "particle-steps/s"
# Algorithmic HBM bytes per particle-step of a separate scan-and-search step (the roofline
# unit): read parent x, y; write x, y; write L; scan (read L, write C); search (read C).
BYTES_PER_PSTEP = {"ref64": 64, "f32": 32, "f16": 20, "bf16": 20}
# The fused step kernel moves less: read L + x, y of the previous frame, write x, y + L of
# the new frame (no CDF or ancestor array goes through memory).
FUSED_BYTES_PER_PSTEP = {"ref64": 48, "f32": 24, "f16": 12, "bf16": 12}
DTYPE_NAME = {"ref64": "f64", "f32": "f32", "f16": "f16", "bf16": "bf16"}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="f16", choices=["ref64", "f32", "f16", "bf16"])
    p.add_argument("--only", action="store_true", help="time the headline precision only")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--frames", type=int, default=T_)
    p.add_argument("--no-batch", action="store_true", help="skip the batched-trackers measurement")
    p.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    p.add_argument("--serve-seconds", type=float, default=20.0,
                   help="length of the served-streams run (the served workload is stated for 60 s; "
                        "20 s by default to keep the bench within a few minutes)")
    p.add_argument("--serve-overload", type=float, default=20.0,
                   help="also replay the served workload with every stream's particle count scaled by this "
                        "factor (capped at 2^24) so that admission refuses streams; 0 = skip")
    p.add_argument("--no-sweep", action="store_true",
                   help="no effect: the sweep runs only with --systems (kept so that older profile command "
                        "lines run unchanged)")
    p.add_argument("--systems", action="store_true",
                   help="also run the precision/size sweep, the paper's workload, the resampler and Gumbel-max "
                        "studies (printed in the detail line on stderr)")
    p.add_argument("--resampler", default="systematic",
                   choices=["systematic", "stratified", "multinomial", "metropolis", "rejection"],
                   help="resampling scheme of the timed filters (the paper's is systematic)")
    p.add_argument("--tpb-sweep", action="store_true",
                   help="thread-block study: build the step kernel at 128/256/512/1024 threads per CTA and time each")
    p.add_argument("--tpb-child", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--core-peaks", action="store_true",
                   help="measure the CUDA-core throughputs (FP32/FP16x2/BF16x2/FP64 FMA, ex2, IMAD, logic, "
                        "shared loads) with the microbenchmark; one JSON object")
    p.add_argument("--profile-target", nargs=5, metavar=("PREC", "N", "SIZE", "RADIUS", "FRAMES"),
                   help="profiling target: step one PREC tracker of N particles through FRAMES frames of a "
                        "SIZE x SIZE synthetic video with disk radius RADIUS, then exit (no timing)")
    p.add_argument("--gumbel", type=int, default=0, metavar="N",
                   help="Gumbel-max study only: time Gumbel-max, systematic and multinomial resampling of "
                        "an N-particle tracker (N <= 2^16) in --precision on the headline video; one JSON object")
    return p.parse_args()


# ---------------------------------------------------------------------------- distributed
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x, device=None):
    """The largest x over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, ms_local, device=None):
    """Whole-job throughput of independent replicas (one per rank, no data-path
    collective): the units all ranks processed over the slowest rank's time.  Returns
    (units per second, slowest time in ms)."""
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    ms = _max_over_ranks(ms_local, device)
    return units_per_rank * ws / (ms * 1e-3), ms


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self, t0=None, t1=None):
        sm, mx, busy, reasons, n_all = [], [], [], set(), 0
        for ts, line in self.lines:
            if t0 is not None and not (t0 <= ts <= t1):
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            n_all += 1
            try:
                s, m, util = float(f[1]), float(f[2]), float(f[9])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
            mx.append(m)
            sm.append(s)
            if util > 0:
                busy.append(util)
        if not mx:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": n_all, "util_median": statistics.median(busy) if busy else 0.0}


# ---------------------------------------------------------------------------- helpers
def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_SOURCES = ("pf_step.cu", "pf_device.cuh", "pf_internal.h")


def _kernel_source_hash():
    """Hash of the sources that define the step kernel (the runtime does not change it)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2308_00763_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _ncu_figure(key, prec):
    """A per-launch figure of the step kernel from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_sha") != _kernel_source_hash():
        return None
    v = d.get(key, {}).get(prec)
    return float(v) if v is not None else None


def _traffic(prec):
    """DRAM bytes per launch of the step kernel (ncu), or None."""
    return _ncu_figure("dram_bytes_per_launch", prec)


def _core_peaks():
    """The committed CUDA-core microbenchmark result (profiles/cuda_core_peaks.json), or None."""
    try:
        with open(os.path.join(ROOT, "profiles", "cuda_core_peaks.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def _issue_view(prec, launch_us, dev):
    """Instruction-issue view of the step kernel: achieved thread instructions per second
    (warp instructions per launch from the committed ncu capture x 32 / launch time)
    against the issue rate of the SMs: 4 schedulers x 32 lanes x SMs x the maximum SM
    clock (nvidia-smi); the measured rate of the integer-logic microbenchmark
    (profiles/cuda_core_peaks.json) is reported beside it."""
    import torch
    warp_instr = _ncu_figure("warp_instructions_per_launch", prec)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", str(dev.index or 0)], capture_output=True, text=True, timeout=20)
        mhz = float(out.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        mhz = None
    peak = sms * 4 * 32 * mhz * 1e6 if mhz else None
    achieved = warp_instr * 32 / (launch_us * 1e-6) if warp_instr else None
    cp = _core_peaks()
    measured = None
    if cp:
        measured = cp.get("rates", {}).get("xor_add", {}).get("thread_instructions_per_s")
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "thread instructions/s",
            "frac": achieved / peak if (achieved and peak) else None,
            "measured_alu_peak": measured,
            "instructions_per_particle_step": warp_instr * 32 / N_ if warp_instr else None,
            "peak_source": "issue: SMs x 4 schedulers x 32 lanes x max SM clock (%s MHz)" % mhz}


def _run_core_peaks():
    """Build and run the CUDA-core microbenchmark; one JSON object on stdout."""
    from paper_2308_00763_gb300 import build as pbuild
    exe = pbuild.build_core_peaks()
    p = subprocess.run([exe, "5"], capture_output=True, text=True, timeout=600)
    if p.returncode != 0:
        sys.stderr.write(p.stderr)
        return p.returncode
    print(p.stdout.strip())
    return 0


def _rmse(a, b):
    import numpy as np
    return float(math.sqrt(np.mean(np.sum((np.asarray(a) - np.asarray(b)) ** 2, axis=1))))


def _config(args, ws):
    """The workload description both arms print (the reference arm times the same workload)."""
    return {"workload": WORKLOAD_SHORT, "precision": args.precision, "resampler": args.resampler,
            "l2": "flushed between timed steps", "parallelism": "replicas" if ws > 1 else "single GPU"}


# ---------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_2308_00763_gb300 import synth
    oracle.build()
    cores = os.cpu_count() or 1
    frames_per_step = 2
    v = synth.make_video(W_, H_, frames_per_step, R_, noise=NOISE_, seed=SEED_)
    init = tuple(v.centres[0])
    for _ in range(args.warmup):
        oracle.track(v.frames, N_, R_, init=init, seed=SEED_, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.track(v.frames, N_, R_, init=init, seed=SEED_, nthreads=cores)
    dt = time.perf_counter() - t0
    val = N_ * frames_per_step * args.steps / dt
    sample = "first %d frames of the workload at full N = 2^20 per step (FP64 oracle, %d threads)" % (
        frames_per_step, cores)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(args, 1),
        "cpu_baseline": {"value": val, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2308_00763_gb300 as pf
    from paper_2308_00763_gb300 import synth
    pf.lib(build_if_missing=True)

    T = args.frames
    v = synth.make_video(W_, H_, T, R_, noise=NOISE_, seed=SEED_)
    init = tuple(v.centres[0])
    frames_dev = torch.from_numpy(v.frames).to(dev)
    frames_pin = torch.from_numpy(v.frames).pin_memory()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    precs = [args.precision] if args.only else ["ref64", "f32", "f16", "bf16"]
    if args.precision in precs:
        precs.remove(args.precision)
    precs.append(args.precision)     # headline last (clock sampling window)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        return _max_over_ranks(x, dev)

    clocks = ClockSampler(local)
    results = {}
    tracks = {}
    for prec in precs:
        f = pf.Filter(W_, H_, N_, R_, prec, init=init, seed=SEED_ + rank, tracker_id=rank, stream=stream,
                      resampler=args.resampler)
        for _ in range(args.warmup):
            f.reset()
            f.run(frames_dev)
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        headline = prec == args.precision
        if headline:
            clocks.start()
            time.sleep(0.3)
        wall0 = time.time()
        for k in range(args.steps):
            flush.zero_()                       # L2 flush, outside the timed events
            ev[k][0].record(stream)
            f.reset()
            f.run(frames_dev)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        wall1 = time.time()
        if headline:
            clocks.stop()
        total_ms = sum(a.elapsed_time(b) for a, b in ev)
        value, total_ms = replica_value(N_ * T * args.steps, total_ms, dev)
        tracks[prec] = f.estimates(0, T)
        # per-launch duration of the step kernel (events between launches on its stream)
        f.reset()
        lev = [torch.cuda.Event(enable_timing=True) for _ in range(T + 1)]
        flush.zero_()
        lev[0].record(stream)
        for t in range(T):
            f.step(frames_dev[t])
            lev[t + 1].record(stream)
        torch.cuda.synchronize(dev)
        launch_ms = [lev[t].elapsed_time(lev[t + 1]) for t in range(T)]
        # end to end: pinned host frames through the C ABI, estimates read back
        barrier()
        e2e_times = []
        for k in range(max(1, min(args.steps, 10))):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            f.reset()
            f.run(frames_pin)
            est = f.estimates(0, T)            # synchronises + D2H of the per-frame estimates
            e2e_times.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(sum(e2e_times)) / len(e2e_times)
        results[prec] = {
            "value": value, "ms_per_step": total_ms / args.steps,
            "launch_us_mean": 1e3 * statistics.mean(launch_ms),
            "launch_us_median": 1e3 * statistics.median(launch_ms),
            # per-frame step latency (one pf_step_frame per frame, device frames)
            "frame_latency_us_p50": 1e3 * statistics.median(launch_ms),
            "frame_latency_us_p99": 1e3 * sorted(launch_ms)[min(len(launch_ms) - 1, int(0.99 * len(launch_ms)))],
            "e2e_value": N_ * T * ws / e2e_s, "wall": (wall0, wall1),
        }
        f.close()
        del est

    # accuracy of every precision against the REF64 GPU track
    ref = tracks.get("ref64")
    for prec in results:
        results[prec]["rmse_px_vs_ref64_gpu"] = _rmse(tracks[prec], ref) if ref is not None else None
    results_truth = {p: _rmse(tracks[p], v.centres) for p in tracks}

    hp = args.precision
    head = results[hp]
    hbm, peak_kind = _peaks()
    # average launch duration of the step kernel over the timed region: the graph-replayed
    # frames of a step, back to back on the filter's stream (gaps between launches included)
    launch_us = 1e3 * head["ms_per_step"] / T
    achieved_gbs = BYTES_PER_PSTEP[hp] * N_ / (launch_us * 1e-6) / 1e9
    fused_gbs = FUSED_BYTES_PER_PSTEP[hp] * N_ / (launch_us * 1e-6) / 1e9
    traffic = _traffic(hp)
    issue = _issue_view(hp, launch_us, dev)
    line = {
        "metric": METRIC, "value": head["value"], "unit": METRIC, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_NAME[hp], "data": "synthetic",
        "config": _config(args, ws),
        # the step kernel against HBM on the scan-and-search design's bytes per particle-step
        # (20 / 32 / 64 B: read x, y, write x, y, write L, scan L -> C, search C); the fused
        # kernel itself moves 12 / 24 / 48 B (fused_frac)
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                     "frac": achieved_gbs / hbm, "traffic": traffic, "kernel": "step_kernel<%s>" % hp,
                     "peak_source": peak_kind, "bytes_per_particle_step": BYTES_PER_PSTEP[hp],
                     "launch_us": launch_us, "fused_frac": fused_gbs / hbm},
        # the same launches against instruction issue (the bound that binds this kernel)
        "roofline_issue": {k: issue[k] for k in ("bound", "frac", "instructions_per_particle_step")},
        "e2e": {"value": head["e2e_value"], "unit": METRIC, "h2d_bytes_per_step": int(W_ * H_ * T),
                "d2h_bytes_per_step": int(16 * T)},
        # multinomial: CDF + pull; Metropolis, rejection: ancestors + pull
        "gpu_launches": args.steps * T * (2 if args.resampler in ("multinomial", "metropolis", "rejection") else 1),
        "accuracy": {"rmse_px_vs_ref64_gpu": head["rmse_px_vs_ref64_gpu"],
                     "rmse_px_vs_ground_truth": results_truth.get(hp)},
        "per_precision": {p: {"value": r["value"], "us_per_frame": 1e3 * r["ms_per_step"] / T}
                          for p, r in results.items()},
    }
    detail = {"per_precision": {p: {k: r[k] for k in ("value", "ms_per_step", "launch_us_median",
                                                      "frame_latency_us_p50", "frame_latency_us_p99",
                                                      "e2e_value", "rmse_px_vs_ref64_gpu")}
                                for p, r in results.items()},
              "roofline_issue": issue, "workload": WORKLOAD}
    cs = clocks.summary(*head["wall"]) or clocks.summary()
    line["clocks"] = {k: cs[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")} if cs else None
    detail["clocks"] = cs
    if not args.no_batch and ws == 1:
        b = _batched(dev, stream, max(3, min(args.steps, 10)), 2, hp)
        detail["batched"] = b
        line["batched"] = {"value": b["value"], "us_per_frame": b["us_per_frame"],
                           "autotuned_value": b["autotuned"]["value"], "trackers": 256}
    if args.systems and ws == 1:
        detail["sweep"] = _sweep(dev, stream)
        detail["paper_workload"] = _paper_workload(dev, stream)
        detail["resamplers"] = _resamplers(dev, stream)
        detail["gumbel_max"] = _gumbel_max(dev, stream)
    if not args.no_serve and ws == 1:
        cap = min(results[p]["value"] for p in results if p in ("f16", "f32")) if any(
            p in results for p in ("f16", "f32")) else head["value"]
        s = _serving(dev, cap, args.serve_seconds, args.serve_overload)
        detail["serving"] = s
        line["serving"] = {"seconds": args.serve_seconds, "streams": 1024,
                           "p50_ms": s["realtime"]["latency_p50_ms"], "p99_ms": s["realtime"]["latency_p99_ms"],
                           "saturated_value": s["saturated"]["value"],
                           "rejected": s["realtime"]["streams_rejected"]}
        if "overloaded" in s:
            o = s["overloaded"]
            line["serving"]["overloaded"] = {"p50_ms": o["latency_p50_ms"], "p99_ms": o["latency_p99_ms"],
                                             "rejected": o["streams_rejected"], "admitted": o["streams_admitted"]}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = _cpu_baseline(v, tracks)
        detail["cpu_baseline"] = cb
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        line["accuracy"]["rmse_px_vs_oracle"] = cb["gpu_rmse_px_vs_oracle"].get(hp)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        # the detail first (stderr), the headline last on stdout, compact
        sys.stderr.write("bench detail: " + json.dumps(detail) + "\n")
        sys.stderr.flush()
        print(json.dumps(_rounded(line), separators=(",", ":")))
    return 0


def _rounded(obj, keep=("value", "ms_per_step")):
    """The headline line with its floats at five significant digits (it must stay short;
    `value` and `ms_per_step` at the top level keep full precision)."""
    def r(x, top=False, key=None):
        if isinstance(x, float) and not (top and key in keep):
            return float("%.5g" % x)
        if isinstance(x, dict):
            return {k: r(v, False, k) for k, v in x.items()}
        if isinstance(x, list):
            return [r(v) for v in x]
        return x
    return {k: r(v, True, k) for k, v in obj.items()}


def _cpu_baseline(v, tracks):
    """The FP64 oracle as it stands, on all host cores, over the whole workload (every frame
    at full N), and the GPU tracks' RMSE against it."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    frames = v.T
    t0 = time.perf_counter()
    est, _, _ = oracle.track(v.frames[:frames], N_, R_, init=tuple(v.centres[0]), seed=SEED_, nthreads=cores)
    dt = time.perf_counter() - t0
    out = {"value": N_ * frames / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
           "sample": "whole workload (%d frames, N = 2^20), %d threads" % (frames, cores),
           "seconds": dt}
    out["gpu_rmse_px_vs_oracle"] = {p: _rmse(tr[:frames], est) for p, tr in tracks.items()}
    return out


def _batched(dev, stream, steps, warmup, precision):
    """256 independent trackers of uneven size (frames 256^2..1024^2, 1k..262k particles,
    radius 3..12, speed < 4 px/frame, 60 frames, sigma 2 px) in one launch per frame, their
    videos resident in HBM, the 60 launches of a step replayed from one CUDA graph; timed
    with the default launch shapes and again with the shape the autotuner picks for this
    batch (its sweep timed on the batch itself)."""
    import numpy as np
    import torch
    import paper_2308_00763_gb300 as pf
    from paper_2308_00763_gb300 import synth
    specs = synth.batch_workload()
    vids = [synth.make_video_device(s["W"], s["H"], s["T"], s["r"], v=s["v"], noise=s["noise"], seed=s["seed"],
                                    device=dev) for s in specs]
    T = specs[0]["T"]
    total_n = sum(s["N"] for s in specs)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def cfgs_for(flags):
        return [pf.make_config(s["W"], s["H"], s["N"], s["r"], precision, init=tuple(c[0]), sigma=(2.0, 2.0),
                               seed=s["seed"], tracker_id=i, flags=flags)
                for i, (s, (_, c)) in enumerate(zip(specs, vids))]

    def timed(cfgs):
        b = pf.Batch(cfgs, stream=stream)
        b.set_videos([f for f, _ in vids])
        for _ in range(warmup):
            b.reset()
            b.run(T)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            b.reset()
            b.run(T)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        ms = [a.elapsed_time(c) for a, c in ev]
        est = np.stack([b.estimates(t) for t in range(T)], axis=1)        # (trackers, T, 2)
        b.close()
        return ms, est

    ms, est = timed(cfgs_for(0))
    err = [float(np.sqrt(np.mean(np.sum((est[i] - vids[i][1]) ** 2, axis=1)))) for i in range(len(specs))]
    out = {"workload": "256 trackers, frames 256^2-1024^2, 1k-262k particles (sum %d), r 3-12, 60 frames" % total_n,
           "precision": precision, "value": total_n * T * steps / (sum(ms) * 1e-3), "unit": METRIC,
           "ms_per_step": sum(ms) / steps, "us_per_frame": 1e3 * sum(ms) / steps / T, "steps": steps,
           "gpu_launches_per_step": T, "rmse_px_vs_truth_median": float(np.median(err)),
           "trackers_within_2px": int(sum(e < 2.0 for e in err))}

    # autotuned shape: the sweep run on this batch itself (8 frames of every video)
    pf.pf_tuning_clear()
    t0 = time.perf_counter()
    shape, us = pf.autotune_batch(cfgs_for(0), [f[:8] for f, _ in vids])
    tune_s = time.perf_counter() - t0
    ms_t, est_t = timed(cfgs_for(pf.PF_FLAG_TUNED))
    err_t = [float(np.sqrt(np.mean(np.sum((est_t[i] - vids[i][1]) ** 2, axis=1)))) for i in range(len(specs))]
    pf.pf_tuning_clear()
    out["autotuned"] = {"value": total_n * T * steps / (sum(ms_t) * 1e-3), "unit": METRIC,
                        "us_per_frame": 1e3 * sum(ms_t) / steps / T, "tuning_seconds": tune_s, "shape": shape,
                        "sweep_best_us_per_frame": us, "rmse_px_vs_truth_median": float(np.median(err_t))}
    del vids
    return out


def _serving(dev, capacity, seconds, overload=0.0):
    """Served multi-camera tracking: 1024 camera streams opening and closing over a run
    of `seconds` (frames 256^2..1024^2, 4k..1M particles, FP16/FP32 half and half, Poisson
    arrivals at 30 fps) replayed through the server's request loop, once in real time
    (per-frame latency from arrival to estimate) and once as fast as the loop runs (the
    served throughput when frames are always waiting).  With `overload` > 0 a third,
    real-time replay (at most 10 s) scales every stream's particle count by that factor
    (capped at 2^24), so that the memory and compute budgets refuse streams.  Frames are
    device-resident 8-frame videos per (size, radius), cycled."""
    import ctypes
    import torch
    import paper_2308_00763_gb300 as pf
    from paper_2308_00763_gb300 import synth
    vids = {}

    def trace(specs, scale):
        for s in specs:
            key = (s["W"], s["r"])
            if key not in vids:
                vids[key] = synth.make_video_device(s["W"], s["H"], 8, s["r"], v=(1.0, -2.0), seed=300 + len(vids),
                                                    device=dev)
        cfgs = [pf.make_config(s["W"], s["H"], min(1 << 24, int(s["N"] * scale)), s["r"], s["precision"],
                               init=tuple(vids[(s["W"], s["r"])][1][0]), seed=s["seed"], tracker_id=i,
                               est_capacity=16) for i, s in enumerate(specs)]
        ev = []
        for i, (s, c) in enumerate(zip(specs, cfgs)):
            fr = vids[(s["W"], s["r"])][0]
            ev.append((s["open"], 0, i, None, 0, ctypes.pointer(c), 30.0))
            for k, t in enumerate(s["arrivals"]):
                ev.append((t, 1, i, fr[k % 8].data_ptr(), fr.stride(1), None, 0.0))
            ev.append((s["close"], 2, i, None, 0, None, 0.0))
        ev.sort(key=lambda e: (e[0], e[1] != 0, e[1] == 2))
        return cfgs, [pf.PfTraceEvent(time_s=e[0], kind=e[1], stream=e[2], frame=e[3], pitch_bytes=e[4], cfg=e[5],
                                      fps=e[6]) for e in ev]

    def replay(specs, events, realtime):
        srv = pf.Server(24 << 30, capacity=capacity, headroom=0.8, max_streams=1024, queue_depth=8, max_in_flight=2)
        t0 = time.perf_counter()
        srv.replay(events, len(specs), realtime=realtime)
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        busy = max(1e-9, st["last_done_s"] - st["first_launch_s"])
        return {"wall_s": wall, "value": st["particle_steps"] / busy, "unit": METRIC,
                "latency_p50_ms": st["latency_p50_ms"], "latency_p99_ms": st["latency_p99_ms"],
                "latency_max_ms": st["latency_max_ms"], "streams_admitted": st["streams_admitted"],
                "streams_rejected": st["streams_rejected"], "frames_done": st["frames_done"],
                "frames_rejected": st["frames_rejected"], "launches": st["launches"],
                "hbm_peak_bytes": st["hbm_peak"]}

    specs = synth.serving_workload(1024, seconds)
    cfgs, events = trace(specs, 1.0)
    torch.cuda.synchronize(dev)
    out = {"workload": "1024 camera streams over %g s: open U(0, %g s), lifetime U(%g s, %g s) clipped, "
                       "frames 256^2-1024^2, N log-uniform 4096-2^20, r 3-12, FP16/FP32 1:1, Poisson 30 fps"
                       % (seconds, seconds * 5 / 6, seconds / 12, seconds),
           "frames_offered": sum(len(s["arrivals"]) for s in specs),
           "particle_steps_offered": float(sum(len(s["arrivals"]) * s["N"] for s in specs)),
           "capacity_admitted": capacity, "headroom": 0.8}
    for mode, realtime in (("realtime", True), ("saturated", False)):
        out[mode] = replay(specs, events, realtime)
    if overload > 0:
        so = min(seconds, 10.0)
        ospecs = synth.serving_workload(1024, so)
        ocfgs, oevents = trace(ospecs, overload)
        out["overloaded"] = replay(ospecs, oevents, True)
        out["overloaded"].update({
            "seconds": so, "particle_scale": overload,
            "demand_all_open": float(sum(30.0 * c.num_particles for c in ocfgs)),
            "particle_steps_offered": float(sum(len(s["arrivals"]) * c.num_particles
                                                for s, c in zip(ospecs, ocfgs)))})
    del vids
    return out


def _sweep(dev, stream):
    """Precision / size sweep: 1024^2 frames, 50 frames, disk radius 10, noise sigma in
    {2, 5, 15} (video seeds 1, 2, 3), N = 2^14 .. 2^24 by powers of 4, REF64 / F32 / F16 /
    BF16 with FP32 accumulation of the likelihood; per run the particle-steps/s of the
    whole track (resident frames, one replayed graph) and the track RMSE against the REF64
    GPU track of the same video and N."""
    import torch
    import paper_2308_00763_gb300 as pf
    from paper_2308_00763_gb300 import synth
    T, W, r = 50, 1024, 10
    runs = []
    for k, noise in enumerate((2.0, 5.0, 15.0)):
        v = synth.make_video(W, W, T, r, noise=noise, seed=k + 1)
        fr = torch.from_numpy(v.frames).to(dev)
        for lg in range(14, 25, 2):
            N = 1 << lg
            ref = None
            for prec in ("ref64", "f32", "f16", "bf16"):
                f = pf.Filter(W, W, N, r, prec, init=tuple(v.centres[0]), seed=k + 1, stream=stream,
                              flags=pf.PF_FLAG_ACCUM32 if prec == "f16" else 0)
                f.run(fr[:4])                                    # warm-up (graph capture)
                f.reset()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                f.run(fr)
                b.record(stream)
                torch.cuda.synchronize(dev)
                ms = a.elapsed_time(b)
                est = f.estimates(0, T)
                f.close()
                if prec == "ref64":
                    ref = est
                runs.append({"noise": noise, "N": N, "precision": prec, "value": N * T / (ms * 1e-3),
                             "us_per_frame": 1e3 * ms / T, "rmse_px_vs_ref64_gpu": _rmse(est, ref),
                             "rmse_px_vs_truth": _rmse(est, v.centres)})
        del fr
    return {"workload": "1024^2 frames, 50 frames, r = 10, noise {2, 5, 15}, N 2^14..2^24 by 4x, "
                        "FP32 accumulation of the likelihood", "unit": METRIC, "runs": runs}


def _paper_workload(dev, stream):
    """The paper's own motion model (drift (1, 2), sigma (5, 2); Eq. 1-2) on a 512^2
    bouncing-disk video of 100 frames at its particle counts (128, 32k, 64k): us per frame
    per precision and the FP16 speedups over FP32 and REF64 (the paper reports 1.5-2x and
    2.5-4.6x on V100 / A100 / A40 / T4; quoted as context, other hardware)."""
    import torch
    import paper_2308_00763_gb300 as pf
    from paper_2308_00763_gb300 import synth
    v = synth.make_video(512, 512, 100, 5, noise=5.0, seed=1, v=(1.0, 2.0))
    fr = torch.from_numpy(v.frames).to(dev)
    out = {}
    for N in (128, 32768, 65536):
        row = {}
        for prec in ("ref64", "f32", "f16"):
            f = pf.Filter(512, 512, N, 5, prec, init=tuple(v.centres[0]), seed=1, stream=stream, sigma=(5.0, 2.0),
                          drift=(1.0, 2.0))
            f.run(fr[:4])
            f.reset()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f.run(fr)
            b.record(stream)
            torch.cuda.synchronize(dev)
            row[prec] = {"us_per_frame": 10.0 * a.elapsed_time(b), "rmse_px_vs_truth": _rmse(f.estimates(0, 100), v.centres)}
            f.close()
        row["speedup_f16_over_f32"] = row["f32"]["us_per_frame"] / row["f16"]["us_per_frame"]
        row["speedup_f16_over_ref64"] = row["ref64"]["us_per_frame"] / row["f16"]["us_per_frame"]
        out[str(N)] = row
    return {"workload": "512^2, 100 frames, disk r = 5 moving (+1, +2), drift (1, 2), sigma (5, 2)", "by_particles": out}


def _resamplers(dev, stream):
    """Systematic (the paper's scheme, Sec. IV) against stratified (one offset per stratum,
    Sec. III), multinomial (independent draws searched in the CDF; CDF and pull kernels),
    Metropolis (64-step chains, Sec. III; chain and pull kernels) and rejection resampling
    (first candidate passing u <= w / w_max, Sec. III; try and pull kernels) on the headline
    workload: us per frame and the track's RMSE against the ground truth, per precision."""
    import torch
    import paper_2308_00763_gb300 as pf
    from paper_2308_00763_gb300 import synth
    v = synth.make_video(W_, H_, T_, R_, noise=NOISE_, seed=SEED_)
    fr = torch.from_numpy(v.frames).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    out = {}
    for prec in ("ref64", "f32", "f16"):
        row = {}
        for rs in ("systematic", "stratified", "multinomial", "metropolis", "rejection"):
            f = pf.Filter(W_, H_, N_, R_, prec, init=tuple(v.centres[0]), seed=SEED_, stream=stream, resampler=rs)
            f.run(fr[:4])
            best = None
            for _ in range(2):
                flush.zero_()
                f.reset()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                f.run(fr)
                b.record(stream)
                torch.cuda.synchronize(dev)
                us = 1e3 * a.elapsed_time(b) / T_
                best = us if best is None else min(best, us)
            row[rs] = {"us_per_frame": best, "value": N_ / (best * 1e-6),
                       "rmse_px_vs_truth": _rmse(f.estimates(0, T_), v.centres)}
            f.close()
        for rs in ("stratified", "multinomial", "metropolis", "rejection"):
            row[rs + "_over_systematic_time"] = row[rs]["us_per_frame"] / row["systematic"]["us_per_frame"]
        out[prec] = row
    return {"workload": WORKLOAD, "unit": METRIC, "by_precision": out}


def _gumbel_max(dev, stream, sizes=None):
    """Gumbel-max resampling (argmax of L + Gumbel variates, Sec. IV's log-domain
    alternative) against systematic and multinomial resampling on the headline video at
    the tracker sizes it allows (N^2 variates a frame): us per frame over 20 frames, and
    the argmax kernel's variate rate (N^2 per frame over the frame time)."""
    import torch
    import paper_2308_00763_gb300 as pf
    from paper_2308_00763_gb300 import synth
    T = 20
    v = synth.make_video(W_, H_, T, R_, noise=NOISE_, seed=SEED_)
    fr = torch.from_numpy(v.frames).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def timed(n, prec, rs):
        f = pf.Filter(W_, H_, n, R_, prec, init=tuple(v.centres[0]), seed=SEED_, stream=stream, resampler=rs)
        f.run(fr[:4])
        best = None
        for _ in range(2):
            flush.zero_()
            f.reset()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f.run(fr)
            b.record(stream)
            torch.cuda.synchronize(dev)
            us = 1e3 * a.elapsed_time(b) / T
            best = us if best is None else min(best, us)
        rmse = _rmse(f.estimates(0, T), v.centres[:T])
        f.close()
        return best, rmse

    out = {}
    if sizes is None:
        sizes = {"ref64": (1000, 4096, 16384), "f32": (1000, 4096, 16384, 65536), "f16": (1000, 4096, 16384, 65536)}
    for prec, ns in sizes.items():
        rows = []
        for n in ns:
            g_us, g_rmse = timed(n, prec, "gumbel")
            s_us, _ = timed(n, prec, "systematic")
            m_us, _ = timed(n, prec, "multinomial")
            rows.append({"N": n, "gumbel_us_per_frame": g_us, "systematic_us_per_frame": s_us,
                         "multinomial_us_per_frame": m_us, "gumbel_variates_per_s": n * n / (g_us * 1e-6),
                         "gumbel_rmse_px_vs_truth": g_rmse})
        out[prec] = rows
    return {"video": "%dx%d, r = %d, %d frames" % (W_, H_, R_, T), "by_precision": out}


def _tpb_child():
    """One study build (selected by PF_STEP_THREADS): us per frame of the headline workload
    (2^20 particles) and of a small tracker (2^16) per precision; one JSON object."""
    import torch
    import paper_2308_00763_gb300 as pf
    from paper_2308_00763_gb300 import synth
    pf.lib(build_if_missing=True)
    dev = torch.device("cuda")
    stream = torch.cuda.Stream()
    v = synth.make_video(W_, H_, T_, R_, noise=NOISE_, seed=SEED_)
    fr = torch.from_numpy(v.frames).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def timed(n, prec, flags=0):
        try:
            f = pf.Filter(W_, H_, n, R_, prec, init=tuple(v.centres[0]), seed=SEED_, stream=stream, flags=flags)
        except RuntimeError as e:           # the 1024-thread build has no REF64 kernel
            return {"unavailable": str(e)}
        f.run(fr[:4])
        best = None
        for _ in range(3):
            flush.zero_()
            f.reset()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f.run(fr)
            b.record(stream)
            torch.cuda.synchronize(dev)
            us = 1e3 * a.elapsed_time(b) / T_
            best = us if best is None else min(best, us)
        r = {"us_per_frame": best, "value": n / (best * 1e-6), "rmse_px_vs_truth": _rmse(f.estimates(0, T_), v.centres)}
        f.close()
        return r

    out = {}
    for n in (N_, 1 << 16):
        out[str(n)] = {prec: timed(n, prec) for prec in ("ref64", "f32", "f16", "bf16")}
    if os.environ.get("PF_STEP_THREADS") == "512":
        # the library's kernel with the tile forced through the tuning cache (the default
        # rule keeps 4096-particle tiles below half a device, which batches prefer)
        tiles = {}
        for n in (1 << 16, 1 << 18, N_):
            for prec in ("ref64", "f32", "f16"):
                for tile in (1024, 2048, 4096):
                    pf.pf_tuning_clear()
                    pf.pf_tuning_store(pf.make_config(W_, H_, n, R_, prec), tile, 0, 0)
                    tiles["%s/%d/%d" % (prec, n, tile)] = timed(n, prec, pf.PF_FLAG_TUNED)["us_per_frame"]
        pf.pf_tuning_clear()
        out["forced_tiles_us_per_frame"] = tiles
    print(json.dumps(out))
    return 0


def _tpb_sweep():
    """Thread-block study (the paper varies threads per block from 32 to 1024): the step
    kernel built at 128, 256, 512 (the library) and 1024 threads per CTA, 8 CDF elements a
    thread, each timed in its own process; one JSON line."""
    import subprocess
    from concurrent.futures import ThreadPoolExecutor
    from paper_2308_00763_gb300 import build as pbuild
    with ThreadPoolExecutor(len(pbuild.STUDY_THREADS)) as ex:
        list(ex.map(lambda t: pbuild.build(threads=t), pbuild.STUDY_THREADS))
    res = {}
    for t in pbuild.STUDY_THREADS:
        env = dict(os.environ, PF_STEP_THREADS=str(t))
        p = subprocess.run([sys.executable, os.path.abspath(__file__), "--tpb-child"], env=env,
                           capture_output=True, text=True, timeout=900)
        if p.returncode != 0:
            res[str(t)] = {"error": (p.stderr or p.stdout).strip().splitlines()[-1:]}
            continue
        res[str(t)] = json.loads(p.stdout.strip().splitlines()[-1])
    print(json.dumps({"study": "threads per CTA of the step kernel", "workload": WORKLOAD, "unit": "us per frame",
                      "particles": [N_, 1 << 16], "by_threads": res}))
    return 0


def _profile_target(prec, n, size, radius, frames):
    """A few frames of one tracker, for an ncu capture of the step kernel at a given size."""
    import torch
    import paper_2308_00763_gb300 as pf
    from paper_2308_00763_gb300 import synth
    n, size, radius, frames = int(n), int(size), int(radius), int(frames)
    v = synth.make_video(size, size, frames, radius, noise=NOISE_, seed=SEED_)
    fr = torch.from_numpy(v.frames).cuda()
    f = pf.Filter(size, size, n, radius, prec, init=tuple(v.centres[0]), seed=SEED_)
    for t in range(frames):
        f.step(fr[t])
    torch.cuda.synchronize()
    print(json.dumps({"profile_target": prec, "N": n, "size": size, "radius": radius, "frames": frames,
                      "last_estimate": f.estimates(frames - 1, 1).tolist()[0]}))
    f.close()
    return 0


def main():
    args = _args()
    if args.tpb_child:
        return _tpb_child()
    if args.tpb_sweep:
        return _tpb_sweep()
    if args.core_peaks:
        return _run_core_peaks()
    if args.profile_target:
        return _profile_target(*args.profile_target)
    if args.gumbel:
        import torch
        print(json.dumps(_gumbel_max(torch.device("cuda"), torch.cuda.Stream(), {args.precision: (args.gumbel,)})))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
