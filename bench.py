"""Benchmark: likelihood evaluations per second inside nested-sampling
iterations on one GB300, in mixed precision, on the largest single-GPU
workload: 3 detectors, 11 parameters, 256 s at 20-2048 Hz (519,169 bins),
2000 live points and 1000 chains of 55 slice steps per iteration.

A step is one ns_step: selection of the 1000 lowest live points, evidence
update, survivors' covariance and Cholesky factor, 1000 slice-sampling chains
(every candidate's TaylorF2 likelihood on the GPU), and the stopping test.
Every timed step is the analysis' first iteration, restored from the
checkpoint taken after ns_init, so that the CPU oracle (--impl reference)
times a sample of exactly the same chains. The whole run to the stopping rule
(time to log Z) and the FP64 form on the same iteration are reported beside
it. Inputs are synthetic and seeded (gwinputs); the injection is made with the
library's own waveform.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (plain FP64 C, all host cores) on a
bounded sample of the same chains. Under torchrun each rank runs an
independent replica (different seeds); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gwinputs as gi  # noqa: E402

METRIC = "logL evals/sec (mixed precision, in nested-sampling iterations)"
UNIT = "evals/s"
WORKLOAD = "c4"
# chains of the first iteration the oracle times per reference step, and the
# slice steps of each it runs (the first ones of the chain: the same draws and
# evaluations the GPU makes at the start of those chains)
REF_CHAINS = 32
REF_STEPS = 2
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
# FP64 pipe peak derived from the unit count: 2 FP64 FMA per clock per SM
# (1.25 TFLOP/s nominal over 152 SMs at 2070 MHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP32_LANE_OPS = 152 * 128 * 2.070e9    # FP32 pipe: 128 lanes/clk/SM x 152 SMs x 2070 MHz
SFU_LANE_OPS = 152 * 16 * 2.070e9      # MUFU (sin, cos): 16 lanes/clk/SM x 152 SMs x 2070 MHz
# sources of the slice-update kernel; a DRAM-traffic summary counts only while
# the hash it records matches these files
KERNEL_SOURCES = ("gwns_slice.cuh", "gwns_device.cuh", "gwns_kernels.cuh")
TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "k_slice_mixed_c4_traffic.md")


def config_dict(ws: int) -> dict:
    """The workload's description, identical in both arms."""
    return {"workload": "c4: 3 detectors, 11 parameters (aligned-spin TaylorF2), 256 s at 20-2048 Hz "
                        "(519,169 bins), chirp mass U[1.1,1.5], SNR 30, n_live=2000, k=1000, 55 slice steps "
                        "per chain, mixed precision; each step is the first nested-sampling iteration "
                        "(restored from the post-initialisation checkpoint)",
            "parallelism": f"replicas{ws}", "l2": "flushed before every timed step (256 MB write)"}


def kernel_source_sha16() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2509_24949_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per slice-update launch from the committed ncu summary, or
    None once the kernel's sources have changed since it was captured."""
    try:
        txt = open(TRAFFIC_SUMMARY).read()
    except OSError:
        return None, None
    m_sha = re.search(r"source_sha16:\s*([0-9a-f]{16})", txt)
    m_b = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", txt)
    m_pb = re.search(r"point_bins_per_launch:\s*([0-9]+)", txt)
    if not (m_sha and m_b) or m_sha.group(1) != kernel_source_sha16():
        return None, None
    return int(m_b.group(1)), (int(m_pb.group(1)) if m_pb else None)


def fp64_flops_per_point_bin(n_det: int) -> float:
    """Algorithmic FP64 work of one point-bin, in flops (2 per FMA-equivalent):
    the phase as 8 basis FMAs, one sine/cosine pair (32 FMA-equivalents,
    measured by instruction count), and per detector the complex product with
    the weighted data and one Horner step of the detector rotation (8)."""
    return 2.0 * (8 + 32 + 8 * n_det)


def world():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def reduce_ranks(dist, total_ms: float, evals: float):
    """Whole-job figures of independent replicas: the slowest rank's timed
    region and the evaluations of all ranks."""
    if not dist:
        return float(total_ms), float(evals)
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(evals)], dtype=torch.float64)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def init_dist(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return dist
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_workload(name=WORKLOAD, seed_offset=0):
    w = gi.workload(name)
    w.seed_sampler += 100 * seed_offset
    w.seed_noise += 100 * seed_offset
    w.seed_injection += 100 * seed_offset
    return w


def workload_data(g, w, stream):
    """Host inputs of a workload: strain (library waveform at the injection,
    plus seeded noise), PSD and detector geometry."""
    probe, th = g.make_analysis(w, precision=g.NS_FP64, n_live=2, k=1, stream=stream.cuda_stream)
    data = probe.waveform(th)
    probe.close()
    psd = np.tile(gi.psd_analytic(w.freqs()), (w.n_det, 1))
    if w.noise:
        data = data + gi.noise(w.seed_noise, psd, w.df)
    pos, xarm, yarm = gi.detectors(w.seed_geometry, w.n_det)
    return dict(data=data, psd=psd, pos=pos, xarm=xarm, yarm=yarm), th


def sampler_on(g, w, inputs, precision, stream, **kw):
    args = dict(kind=w.kind, lo=w.lo, hi=w.hi, f0=w.f0, df=w.df, n_live=w.n_live, k=w.k,
                steps_per_dim=w.steps_per_dim, precision=precision, seed=w.seed_sampler,
                stream=stream.cuda_stream, **inputs)
    args.update(kw)
    return g.Sampler(**args)


def timed_first_iterations(sp, blob, stream, steps, flush):
    """`steps` repetitions of the analysis' first iteration (restore, L2
    flush, then CUDA events on the library's stream around ns_step); returns
    per-step ms and the counters' differences over the timed steps."""
    import torch
    ms = []
    evals, pbins, pbins_lo, kern = 0, 0, 0, [0.0] * 5
    for _ in range(steps):
        sp.restore(blob)
        s0 = sp.stats()
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sp.step()
        b.record(stream)
        b.synchronize()
        s1 = sp.stats()
        ms.append(a.elapsed_time(b))
        evals += s1["evals"] - s0["evals"]
        pbins += s1["point_bins"] - s0["point_bins"]
        pbins_lo += s1["point_bins_lo"] - s0["point_bins_lo"]
        kern = [x + (q - p) for x, p, q in zip(kern, s0["kernel_ms"], s1["kernel_ms"])]
    return ms, evals, pbins, kern, pbins_lo


def run_gpu(args):
    import torch
    ws, rank = world()
    dist = init_dist(ws)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.cuda.current_device()
    import paper_2509_24949_gb300 as g
    from paper_2509_24949_gb300 import _build
    if not _build.up_to_date():
        _build.build()
    stream = torch.cuda.Stream()
    w = build_workload(WORKLOAD, rank)
    inputs, th_inj = workload_data(g, w, stream)
    sp = sampler_on(g, w, inputs, g.NS_MIXED, stream)
    blob = sp.checkpoint()          # the initial live set: every timed step starts here
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush():
        with torch.cuda.stream(stream):
            l2_flush.fill_(1.0)

    timed_first_iterations(sp, blob, stream, args.warmup, flush)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        step_ms, evals, pbins, kern, pbins_lo = timed_first_iterations(sp, blob, stream, args.steps, flush)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = sum(step_ms)
    total_ms_max, evals_all = reduce_ranks(dist, total_ms, evals)
    value = evals_all / (total_ms_max / 1e3)
    tile = sp.stats()["mixed_tile"]
    roof = mixed_slice_roofline(kern, pbins, evals, args.steps, w.n_det, tile, sum(kern), pbins_lo)

    extras = rank == 0 and not args.core_only
    # the whole run to the stopping rule, from the same initial state
    ttl = time_to_logz_from(sp, blob) if extras else None
    sp.close()
    # the FP64 form on the same first iteration (one step: ~9 s on this grid)
    fp64 = fp64_first_iteration(g, w, inputs, stream, flush) if extras else None
    # end to end through the C ABI with host buffers
    e2e = e2e_run(g, w, inputs, args.steps, stream)

    serving = serving_stream(g) if extras else None
    agreement = precision_agreement(g, build_workload("c1"), stream, name="c1") if extras else None
    agreement_c4 = per_point_agreement(g, w, inputs, stream, points=1024) if extras else None
    c1 = c1_fp64_extra(g, stream, args.steps, flush) if extras else None
    # the mixed batched likelihood on the same grid (8192 prior draws, three launches)
    mixed_lik = mixed_likelihood_roofline(g, stream) if extras else None

    if rank == 0:
        cpu = cpu_baseline() if ws == 1 and not args.core_only else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded noise, TaylorF2 injection at SNR 30, seeded detectors)",
            "config": config_dict(ws),
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "evals_per_step": evals / args.steps, "point_bins_per_s": pbins / (total_ms / 1e3),
            "time_to_logZ": ttl,
            "fp64_same_iteration": fp64,
            "e2e": e2e,
            "gpu_launches": 5 * args.steps,   # the 5 library kernels of each ns_step (the L2 flush fill is torch's)
            "kernel_ms_per_step": [x / args.steps for x in kern],
            "roofline": roof,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "mixed_vs_fp64": {"c4_per_point": agreement_c4, "c1": agreement},
            "c1_fp64": c1,
            "mixed_likelihood": mixed_lik,
            "serving": serving,
        }
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def executed_count(pb, pb_lo, n_det, tile):
    """FP32 instructions per point-bin the rotation form executes when the
    tile groups from the low-degree threshold run the Taylor degree 3: the
    frozen count less the 4 Horner steps of C_4..C_7 on those bins."""
    return mixed_fp32_per_point_bin(n_det, tile) - LOW_DEGREE_SAVING * (pb_lo / pb if pb else 0.0)


def mixed_slice_roofline(kern, pbins, evals, steps, n_det, tile, step_kernel_ms, pbins_lo=0):
    """Roofline of the fused slice update (k_slice<MIXED>) over the timed
    steps: its average launch duration from the CUDA events recorded around
    it inside the iteration's graph (on the library's stream), and its
    algorithmic instruction count = point-bins processed (device-side count of
    jcut+1 per evaluation) x the binding pipe's instructions per point-bin
    (the count frozen for the degree-7 tiles); beside it the fraction at the
    count the kernel executes (degree 3 on the bins counted in pbins_lo)."""
    ms = kern[3] / steps
    pb = pbins / steps
    frac, pipe = mixed_roofline(pb, ms / 1e3, n_det, tile)
    per_pb = mixed_fp32_per_point_bin(n_det, tile) if pipe == "FP32" else mixed_mufu_per_point_bin(n_det, tile)
    peak = (FP32_LANE_OPS if pipe == "FP32" else SFU_LANE_OPS) / 1e12
    traffic, traffic_pb = recorded_traffic()
    if traffic is not None and traffic_pb:
        traffic = traffic * pb / traffic_pb     # scaled to this launch's point-bins
    return {"bound": "alu", "kernel": f"k_slice_ws<MIXED,{n_det} det> (work-shared fused slice update + likelihood)",
            "pipe": pipe, "achieved": pb * per_pb / (ms / 1e3) / 1e12, "peak": peak,
            "unit": f"T {pipe} lane-instructions/s", "frac": frac,
            "traffic": traffic,
            "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, scaled by "
                            "point-bins; null when the kernel's sources changed since the capture",
            "peak_source": "derived (not measured): 128 FP32 / 16 MUFU lanes/clk/SM x 152 SMs x 2070 MHz",
            "per_launch": {"ms": ms, "evals": evals / steps, "point_bins": pb,
                           "instr_per_point_bin": per_pb, "tile": tile,
                           "share_of_step_kernels": kern[3] / step_kernel_ms if step_kernel_ms else None},
            "at_executed_count": executed_roofline(pb, pbins_lo / steps, ms / 1e3, n_det, tile, pipe)}


def executed_roofline(pb, pb_lo, seconds, n_det, tile, pipe):
    """The FP32 fraction at the instruction count the kernel executes (fewer
    than the frozen count on the bins of the low-degree tile groups)."""
    if pipe != "FP32":
        return None
    per = executed_count(pb, pb_lo, n_det, tile)
    return {"instr_per_point_bin": per, "low_degree_share": pb_lo / pb if pb else 0.0,
            "achieved": pb * per / seconds / 1e12, "frac": pb * per / seconds / FP32_LANE_OPS}


def time_to_logz_from(sp, blob):
    """The whole run from the initial state to the stopping rule (first ns_step
    to ns_result), with per-step latencies."""
    import torch
    sp.restore(blob)
    torch.cuda.synchronize()
    s0 = sp.stats()
    t0 = time.perf_counter()
    ms, done, it = [], False, 0
    while not done and it < 100000:
        t = time.perf_counter()
        done = sp.step()
        ms.append((time.perf_counter() - t) * 1e3)
        it += 1
    r = sp.result(samples=False)
    t1 = time.perf_counter()
    s1 = sp.stats()
    ev = s1["evals"] - s0["evals"]
    return {"seconds": t1 - t0, "iterations": it, "evals": ev, "evals_per_s": ev / (t1 - t0),
            "logZ": r["logZ"], "dlogZ": r["dlogZ"], "p50_step_ms": float(np.percentile(ms, 50)),
            "p99_step_ms": float(np.percentile(ms, 99)), "precision": "mixed",
            "note": "ns_step to ns_result on the host clock, setup excluded"}


def fp64_first_iteration(g, w, inputs, stream, flush):
    """The FP64 form on the same grid: its first iteration timed with CUDA
    events (one step; the FP64 pipe makes it ~40x slower than mixed here)."""
    import torch
    sp = sampler_on(g, w, inputs, g.NS_FP64, stream)
    blob = sp.checkpoint()
    ms, ev, pb, kern, _ = timed_first_iterations(sp, blob, stream, 1, flush)
    sp.close()
    t = sum(ms) / 1e3
    return {"evals_per_s": ev / t, "ms_per_step": sum(ms), "evals": ev, "point_bins_per_s": pb / t,
            "k_slice_frac_fp64_pipe": pb * fp64_flops_per_point_bin(w.n_det) / (kern[3] / 1e3) / (FP64_PEAK_TFLOPS * 1e12),
            "note": "first iteration, one step, CUDA events; FP64 peak derived (2 FMA/clk/SM)"}


def per_point_agreement(g, w, inputs, stream, points=1024):
    """Mixed against FP64 log L on prior draws of a workload's grid."""
    a = sampler_on(g, w, inputs, g.NS_FP64, stream, n_live=8, k=4)
    b = sampler_on(g, w, inputs, g.NS_MIXED, stream, n_live=8, k=4)
    u = gi.unit_cube(777, points, w.dim)
    l64, lmx = a.eval_lnl(u), b.eval_lnl(u)
    a.close()
    b.close()
    d = np.abs(lmx - l64)
    return {"workload": w.name, "points": points, "max_abs_dlogL": float(d.max()),
            "rms_dlogL": float(np.sqrt(np.mean(d * d))), "max_abs_logL": float(np.max(np.abs(l64)))}


def c1_fp64_extra(g, stream, steps, flush):
    """The 4017-bin FP64 workload (the previous headline): K iterations after
    three warm-up iterations of one run, CUDA events, L2 flushed."""
    import torch
    w = build_workload("c1")
    sp, th = g.make_analysis(w, precision=g.NS_FP64, stream=stream.cuda_stream)
    for _ in range(3):
        sp.step()
    s0 = sp.stats()
    ms = []
    for _ in range(steps):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sp.step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    s1 = sp.stats()
    sp.close()
    ttl = {}
    for name, prec in (("fp64", g.NS_FP64), ("mixed", g.NS_MIXED)):
        ttl[name] = time_to_logz(g, w, prec, stream)
    return {"workload": "c1: 3 detectors, 4017 bins, n_live=1000, k=500, FP64",
            "evals_per_s": (s1["evals"] - s0["evals"]) / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps,
            "time_to_logZ": ttl}


def mixed_likelihood_roofline(g, stream):
    """The mixed batched likelihood (`ns_eval_lnl`, kernel k_eval) on the c4
    grid: throughput and the fraction of its binding pipe (derived peaks, as
    for the mixed rows of the table)."""
    r = batch_eval_row(g, "c4", g.NS_MIXED, stream, points=8192, reps=3)
    peak = FP32_LANE_OPS if r["pipe"] == "FP32" else SFU_LANE_OPS
    at_exec = executed_roofline(r["point_bins"], r["point_bins_lo"], r["seconds"], 3, r["mixed_tile"], r["pipe"])
    return {"workload": "c4: 3 detectors, 20-2048 Hz at df=1/256 (519,169 bins), 8192 prior draws, "
                        "mixed precision, 128-bin tiles", "kernel": "k_eval<MIXED,3 det>",
            "evals_per_s": r["batch_evals_per_s"], "point_bins_per_s": r["point_bins_per_s"],
            "bound": r["pipe"], "frac": r["frac"], "peak_lane_ops_per_s": peak,
            "instr_per_point_bin": (mixed_fp32_per_point_bin(3, r["mixed_tile"]) if r["pipe"] == "FP32"
                                    else mixed_mufu_per_point_bin(3, r["mixed_tile"])),
            "peak_source": "derived (not measured): 128 FP32 / 16 MUFU lanes/clk/SM x 152 SMs x 2070 MHz",
            "at_executed_count": at_exec}


def time_to_logz(g, w, precision, stream):
    import torch
    t0 = time.perf_counter()
    sp, _ = g.make_analysis(w, precision=precision, stream=stream.cuda_stream)
    t_setup = time.perf_counter() - t0
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    it = sp.run()
    r = sp.result(samples=False)
    t2 = time.perf_counter()
    s = sp.stats()
    sp.close()
    return {"seconds": t2 - t1, "setup_s": t_setup, "iterations": it, "evals": s["evals"],
            "evals_per_s": s["evals"] / (t2 - t1), "logZ": r["logZ"], "dlogZ": r["dlogZ"]}


def analysis_inputs(g, w, stream):
    """Host inputs of a workload and its (possibly narrowed) prior: the
    single-detector workload fixes its distance from the target SNR."""
    if w.dl_from_snr or w.ideal:
        probe, th = g.make_analysis(w, precision=g.NS_FP64, n_live=2, k=1, stream=stream.cuda_stream)
        data = probe.waveform(th)
        probe.close()
        w2 = gi.workload(w.name)
        w2.seed_sampler = w.seed_sampler
        w2.lo, w2.hi = w.lo.copy(), w.hi.copy()
        w2.lo[gi.P_DL] = w2.hi[gi.P_DL] = th[gi.P_DL]
        psd = np.tile(gi.psd_analytic(w.freqs()), (w.n_det, 1))
        return w2, dict(data=data, psd=psd, ideal=True), th
    inputs, th = workload_data(g, w, stream)
    return w, inputs, th


def precision_agreement(g, w, stream, seeds: int = 16, points: int = 4096, name: str = WORKLOAD):
    """Mixed against FP64 on the GPU: per-point log L difference on prior
    draws, and log Z over `seeds` sampler seeds on the same data (seed pair i:
    both forms with sampler seed + 1000 (i + 1)), reported as the mean
    difference with its standard error."""
    w = gi.workload(name)
    w, inputs, th = analysis_inputs(g, w, stream)
    agree = per_point_agreement(g, w, inputs, stream, points=points)
    if seeds < 2:
        return {"workload": name, "points": points, **{k: agree[k] for k in
                                                       ("max_abs_dlogL", "rms_dlogL", "max_abs_logL")}}
    dz, z64, zmx, dl64 = [], [], [], []
    base = w.seed_sampler
    for i in range(seeds):
        zs = []
        for prec in (g.NS_FP64, g.NS_MIXED):
            sp = sampler_on(g, w, inputs, prec, stream, seed=base + 1000 * (i + 1))
            sp.run()
            r = sp.result(samples=False)
            zs.append(r["logZ"])
            if prec == g.NS_FP64:
                dl64.append(r["dlogZ"])
            sp.close()
        dz.append(zs[1] - zs[0])
        z64.append(zs[0])
        zmx.append(zs[1])
    dz = np.array(dz)
    return {"workload": name, "points": points, "max_abs_dlogL": agree["max_abs_dlogL"],
            "rms_dlogL": agree["rms_dlogL"], "max_abs_logL": agree["max_abs_logL"],
            "seeds": seeds, "mean_dlogZ": float(dz.mean()), "stderr_dlogZ": float(dz.std(ddof=1) / np.sqrt(seeds)),
            "sd_dlogZ_pairs": float(dz.std(ddof=1)),
            "max_abs_dlogZ_single_seed": float(np.abs(dz).max()),
            "mean_logZ_fp64": float(np.mean(z64)), "mean_logZ_mixed": float(np.mean(zmx)),
            "sd_logZ_fp64_over_seeds": float(np.std(z64, ddof=1)),
            "sd_logZ_mixed_over_seeds": float(np.std(zmx, ddof=1)),
            "mean_dlogZ_reported_fp64": float(np.mean(dl64))}


def e2e_run(g, w, inputs, steps, stream):
    """The headline metric end to end through the C ABI with host buffers:
    ns_init from host arrays (strain and PSD uploaded, tables built, the
    initial live set drawn and evaluated), then per step ns_restore from a
    pinned host checkpoint of the initial state (its live set and run state
    copied host -> device) and ns_step_host (the step's dead points copied
    device -> host into pinned buffers); evaluations of the steps over the
    wall time of all of it."""
    import ctypes
    import torch
    probe = sampler_on(g, w, inputs, g.NS_MIXED, stream)
    blob = probe.checkpoint()
    probe.close()
    hblob = torch.frombuffer(bytearray(blob), dtype=torch.uint8).pin_memory()
    k, d = w.k, w.dim
    du = torch.empty((k, d), dtype=torch.float64).pin_memory()
    dl = torch.empty(k, dtype=torch.float64).pin_memory()
    dw = torch.empty(k, dtype=torch.float64).pin_memory()
    done = ctypes.c_int(0)
    L = g.lib()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sp = sampler_on(g, w, inputs, g.NS_MIXED, stream)
    ev = 0
    for _ in range(steps):
        g._check(L.ns_restore(sp._ctx, hblob.data_ptr(), hblob.numel()), "ns_restore")
        e0 = sp.stats()["evals"]
        g._check(L.ns_step_host(sp._ctx, k, ctypes.byref(done), du.data_ptr(), dl.data_ptr(), dw.data_ptr()),
                 "ns_step_host")
        ev += sp.stats()["evals"] - e0
    t1 = time.perf_counter()
    sp.close()
    init_h2d = (2 * inputs["data"].size + inputs["psd"].size) * 8
    return {"value": ev / (t1 - t0), "unit": UNIT,
            "h2d_bytes_per_step": hblob.numel() + init_h2d / steps,
            "d2h_bytes_per_step": k * (d + 2) * 8,
            "note": "ns_init from host arrays (strain and PSD upload amortised over the steps) + per step "
                    "ns_restore of the pinned initial checkpoint and ns_step_host into pinned buffers"}


def serving_stream(g, count=64, time_limit_s=240.0, max_chains=0):
    """The serving workload: `count` analyses arriving as a Poisson stream at
    2/s (durations 4-64 s at 20-2048 Hz, n_live U{500..2000}, k = n/2, SNR
    U[10, 40], 3 detectors, mixed precision), served by one ns_server that
    interleaves the running analyses' iterations. Arrival -> result latency
    per analysis (p50/p99) and the aggregate likelihood throughput."""
    stream = gi.serving_stream(count=count)
    reqs = []
    for i, r in enumerate(stream):
        w = gi.workload("c3", duration=r["duration"], n_live_c3=r["n_live"], snr_c3=r["snr"])
        w.seed_noise += 10 * i
        w.seed_injection += 10 * i
        w.seed_sampler += 10 * i
        sp, th = g.make_analysis(w, precision=g.NS_MIXED, n_live=2, k=1)
        f = w.freqs()
        psd = np.tile(gi.psd_analytic(f), (w.n_det, 1))
        data = sp.waveform(th) + gi.noise(w.seed_noise, psd, w.df)
        sp.close()
        pos, xarm, yarm = gi.detectors(w.seed_geometry, w.n_det)
        reqs.append((r["arrival_s"], dict(kind=w.kind, lo=w.lo, hi=w.hi, data=data, psd=psd, f0=w.f0, df=w.df,
                                          pos=pos, xarm=xarm, yarm=yarm, n_live=w.n_live, k=w.k,
                                          steps_per_dim=w.steps_per_dim, seed=w.seed_sampler)))
    srv = g.Server(precision=g.NS_MIXED, max_active=16, max_chains=max_chains)
    ids, arrival = [], []
    t0 = srv.time()
    nxt = 0
    while True:
        t = srv.time() - t0
        while nxt < len(reqs) and reqs[nxt][0] <= t:
            ids.append(srv.submit(**reqs[nxt][1]))
            arrival.append(reqs[nxt][0])
            nxt += 1
        r, p = srv.tick()
        if r == 0 and p == 0:
            if nxt == len(reqs):
                break
            time.sleep(max(0.0, min(0.05, reqs[nxt][0] - (srv.time() - t0))))
        if srv.time() - t0 > time_limit_s:
            break
    t_end = srv.time() - t0
    lat, evals, logz = [], 0, []
    for rid, ta in zip(ids, arrival):
        st = srv.poll(rid)
        if st["state"] == g.NS_REQ_DONE:
            lat.append(st["t_done"] - t0 - ta)
            evals += st["evals"]
            logz.append(st["logZ"])
    srv.close()
    return {"requests": count, "completed": len(lat), "makespan_s": t_end,
            "p50_time_to_logZ_s": float(np.percentile(lat, 50)) if lat else None,
            "p99_time_to_logZ_s": float(np.percentile(lat, 99)) if lat else None,
            "evals_per_s": evals / t_end if t_end > 0 else None,
            "workload": "Poisson arrivals at 2/s; durations {4,8,16,32,64} s at 20-2048 Hz "
                        "(8,113-129,793 bins); n_live U{500..2000}, k = n/2; SNR U[10,40]; 3 detectors; "
                        "mixed precision; up to 16 analyses interleaved"}


def oracle_first_iteration():
    """The oracle's own first iteration of the workload: its data (oracle
    waveform, the same seeded noise), the initial live set of the same Philox
    draws evaluated by its per-bin likelihood, the selection and the
    survivors' Cholesky factor (setup of the CPU samples; not timed)."""
    if not hasattr(oracle_first_iteration, "cache"):
        import oracle
        from oracle import ns as ons
        w = build_workload(WORKLOAD)
        pb, th = oracle.make_problem(w)
        st0 = ons.initial_state(pb, w.n_live, w.seed_sampler)
        order = np.argsort(st0.live_logl, kind="stable")
        k = w.k
        surv = np.ascontiguousarray(st0.live_u[order[k:]])
        surv_l = np.ascontiguousarray(st0.live_logl[order[k:]])
        chol = np.ascontiguousarray(ons.survivor_cholesky(surv))
        lstar = float(st0.live_logl[order[k - 1]])
        oracle_first_iteration.cache = (w, pb, surv, surv_l, chol, lstar)
    return oracle_first_iteration.cache


def oracle_chains(first: int):
    """One bounded sample on the oracle: chains first .. first + REF_CHAINS - 1
    (mod k) of the first iteration, each for its first REF_STEPS slice steps --
    the same draws and evaluations the GPU makes at the start of those chains
    in every timed step. Returns (evaluations, seconds, threads)."""
    import oracle
    w, pb, surv, surv_l, chol, lstar = oracle_first_iteration()
    k, d = w.k, pb.dim
    first %= k
    count = min(REF_CHAINS, k - first)
    new_u = np.zeros((k, d))
    new_l = np.zeros(k)
    caps = np.zeros(1, dtype=np.int32)
    nt = oracle.max_threads()
    t0 = time.perf_counter()
    ev = oracle.lib().or_evolve_chains(pb.c, nt, w.seed_sampler, 0, first, count, oracle._ptr(surv),
                                       oracle._ptr(surv_l), w.n_live - k, oracle._ptr(chol), lstar,
                                       REF_STEPS, 64, 64, oracle._ptr(new_u), oracle._ptr(new_l),
                                       oracle._ptr(caps))
    return ev, time.perf_counter() - t0, nt


def ref_sample_text() -> str:
    return (f"per sample: {REF_CHAINS} chains of the first iteration of c4 (a different block of chains each "
            f"time), their first {REF_STEPS} of 55 slice steps (the evaluations the GPU makes first in those "
            f"chains); plain FP64 C with per-bin libm transcendentals, OpenMP over chains")


def cpu_baseline(target_s: float = 12.0):
    """The oracle's chain work of the timed iteration, in bounded samples,
    until about target_s seconds of wall time on all host cores."""
    tot_ev, tot_s, reps, nt = 0, 0.0, 0, 1
    while tot_s < target_s and reps < 200:
        ev, sec, nt = oracle_chains(REF_CHAINS * reps)
        tot_ev += ev
        tot_s += sec
        reps += 1
    return {"value": tot_ev / tot_s, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"{reps} samples ({tot_ev} evaluations, {tot_s:.1f} s); " + ref_sample_text()}


def run_reference(args):
    """The oracle as the reference arm: each step is one bounded sample of the
    timed iteration's chains (a different block of chains per step)."""
    ws, rank = world()
    if rank != 0:
        return
    oracle_first_iteration()
    for i in range(args.warmup):
        oracle_chains(REF_CHAINS * (args.steps + i))
    tot_ev, tot_s, nt = 0, 0.0, 1
    for i in range(args.steps):
        ev, sec, nt = oracle_chains(REF_CHAINS * i)
        tot_ev += ev
        tot_s += sec
    value = tot_ev / tot_s
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded noise, TaylorF2 injection at SNR 30, seeded detectors)",
           "config": config_dict(ws),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                            "sample": ref_sample_text()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# Horner steps the Taylor degree 3 saves per bin against degree 7 (C_4..C_7)
LOW_DEGREE_SAVING = 4.0


def mixed_fp32_per_point_bin(n_det: int, tile: int) -> float:
    """FP32 instructions of the mixed form per point-bin (per-tile or per-flush
    work not counted). Tiles of 32 bins or more: x and x^2 (2), C_1 x as an
    error-free product (3), the Horner sum of C_2..C_7 (6), the reduction of
    C_1 x (2), detector 0's phase in radians (3) and complex MAC (4); per
    further detector the product of the weighted data with detector 0's phasor
    (4), one step of the Horner sum in its rotation (4) and an eighth of a
    segment step (6). Shorter tiles: the common part (12) and per detector
    4 (phase) + 2 (reduction) + 1 (scale) + 4 (complex MAC). Per-bin form
    (tile 0): the double-float dot product of 8 basis terms (12 each) and per
    detector the double-float delay term, reduction and MAC (20)."""
    if tile >= 32:
        return 20.0 + 8.75 * (n_det - 1)
    if tile:
        return 12.0 + 11.0 * n_det
    return 96.0 + 20.0 * n_det


def mixed_mufu_per_point_bin(n_det: int, tile: int) -> float:
    """MUFU instructions (sine, cosine) per point-bin: detector 0's pair on
    tiles of 32 bins or more (the rotated detectors take one pair per tile),
    otherwise a pair per detector."""
    return 2.0 if tile >= 32 else 2.0 * n_det


def mixed_roofline(point_bins: float, seconds: float, n_det: int, tile: int):
    """Fraction of the binding pipe (FP32 or MUFU) the mixed form reaches: the
    time the algorithmic instructions need on that pipe over the measured."""
    t32 = point_bins * mixed_fp32_per_point_bin(n_det, tile) / FP32_LANE_OPS
    tsfu = point_bins * mixed_mufu_per_point_bin(n_det, tile) / SFU_LANE_OPS
    return (t32 / seconds, "FP32") if t32 >= tsfu else (tsfu / seconds, "SFU")


def _timed_steps(sp, stream, max_steps):
    """ns_step until done (or max_steps), each bracketed by CUDA events on the
    library's stream; returns (per-step ms, iterations, done)."""
    import torch
    ms, done, it = [], False, 0
    while not done and it < max_steps:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        done = sp.step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        it += 1
    return ms, it, done


def _rb_analysis(g, w, precision, stream, coarse_bins=1024):
    """The workload's data on the full grid, sampled on coarse relative-binning
    bins about the injection (the fiducial point)."""
    probe, th = g.make_analysis(w, precision=g.NS_FP64, n_live=2, k=1, stream=stream.cuda_stream)
    data = probe.waveform(th)
    probe.close()
    if w.noise:
        data = data + gi.noise(w.seed_noise, np.tile(gi.psd_analytic(w.freqs()), (w.n_det, 1)), w.df)
    return g.sampler_for_workload(w, data=data, precision=precision, coarse_bins=coarse_bins, theta_fid=th,
                                  stream=stream.cuda_stream), th


def table_row(g, name, precision, stream, max_steps=100000, coarse=False):
    import torch
    w = gi.workload(name)
    t0 = time.perf_counter()
    if coarse:
        sp, th = _rb_analysis(g, w, precision, stream)
    else:
        sp, th = g.make_analysis(w, precision=precision, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    st0 = sp.stats()
    t1 = time.perf_counter()
    ms, it, done = _timed_steps(sp, stream, max_steps)
    r = sp.result(samples=False) if done else None
    t2 = time.perf_counter()
    st1 = sp.stats()
    sp.close()
    ev = st1["evals"] - st0["evals"]
    pb = st1["point_bins"] - st0["point_bins"]
    slice_ms = st1["kernel_ms"][3] - st0["kernel_ms"][3]
    if coarse:
        frac, pipe = None, None     # relative-binning sums, not the per-bin work these counts describe
    elif precision == g.NS_FP64:
        frac = pb * fp64_flops_per_point_bin(w.n_det) / (slice_ms / 1e3) / (FP64_PEAK_TFLOPS * 1e12)
        pipe = "FP64"
    else:
        frac, pipe = mixed_roofline(pb, slice_ms / 1e3, w.n_det, st1["mixed_tile"])
    exe = None
    if not coarse and precision != g.NS_FP64 and pb:
        exe = executed_roofline(pb, st1["point_bins_lo"] - st0["point_bins_lo"], slice_ms / 1e3, w.n_det,
                                st1["mixed_tile"], pipe)
    return {"config": name + (" (1024 coarse bins)" if coarse else ""),
            "form": "fp64" if precision == g.NS_FP64 else "mixed", "iterations": it, "done": done,
            "evals": ev, "evals_per_s": ev / (sum(ms) / 1e3), "point_bins_per_s": pb / (sum(ms) / 1e3),
            "bins_per_eval": pb / max(ev, 1), "k_slice_frac": frac, "k_slice_pipe": pipe,
            "k_slice_at_executed_count": exe,
            "mixed_tile": st1["mixed_tile"] if precision != g.NS_FP64 and not coarse else None,
            "time_to_logZ_s": (t2 - t1) if done else None, "setup_s": setup_s,
            "p50_step_ms": float(np.percentile(ms, 50)), "p99_step_ms": float(np.percentile(ms, 99)),
            "logZ": r["logZ"] if r else None, "dlogZ": r["dlogZ"] if r else None}


def batch_eval_row(g, name, precision, stream, points=2048, reps=3, warps=0):
    """Batched likelihood throughput (ns_eval_lnl on prior draws): CUDA events
    on the library's stream around `reps` launches after one warm-up; the
    point-bins come from the library's own count of the bins each point read.
    warps: warps per point (0: the library's choice)."""
    import torch
    w = gi.workload(name)
    sp, th = g.make_analysis(w, precision=precision, n_live=8, k=4, stream=stream.cuda_stream,
                             warps_per_point=warps)
    u = torch.tensor(gi.unit_cube(99, points, w.dim), dtype=torch.float64, device="cuda")
    out = torch.empty(points, dtype=torch.float64, device="cuda")
    sp.eval_lnl(u, out)
    st0 = sp.stats()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        for _ in range(reps):
            g.lib().ns_eval_lnl(sp._ctx, u.data_ptr(), points, out.data_ptr())
        b.record(stream)
    b.synchronize()
    t = a.elapsed_time(b) / 1e3
    st1 = sp.stats()
    sp.close()
    pb = st1["batch_point_bins"] - st0["batch_point_bins"]
    row = {"config": name, "form": "fp64" if precision == g.NS_FP64 else "mixed", "batch_points": points,
           "warps_per_point": warps or None, "seconds": t, "point_bins": pb,
           "point_bins_lo": st1["batch_point_bins_lo"] - st0["batch_point_bins_lo"],
           "batch_evals_per_s": points * reps / t, "point_bins_per_s": pb / t, "bins_per_eval": pb / (points * reps)}
    if precision == g.NS_FP64:
        row["frac"], row["pipe"] = pb * fp64_flops_per_point_bin(w.n_det) / t / (FP64_PEAK_TFLOPS * 1e12), "FP64"
    else:
        row["frac"], row["pipe"] = mixed_roofline(pb, t, w.n_det, st1["mixed_tile"])
        row["mixed_tile"] = st1["mixed_tile"]
    return row


def oracle_rate(name: str, chains: int, steps_per_dim: int, target_s: float):
    """Oracle evaluations per second inside slice-sampling chains of a
    workload's first iteration (plain FP64 C, OpenMP over chains)."""
    import oracle
    from oracle import ns as ons
    w = gi.workload(name)
    pb, th = oracle.make_problem(w)
    st0 = ons.initial_state(pb, w.n_live, w.seed_sampler)
    order = np.argsort(st0.live_logl, kind="stable")
    k, d = w.k, pb.dim
    surv = np.ascontiguousarray(st0.live_u[order[k:]])
    surv_l = np.ascontiguousarray(st0.live_logl[order[k:]])
    chol = np.ascontiguousarray(ons.survivor_cholesky(surv))
    lstar = float(st0.live_logl[order[k - 1]])
    nt = oracle.max_threads()
    tot_ev, tot_s, rep = 0, 0.0, 0
    while tot_s < target_s:
        new_u, new_l = np.zeros((chains, d)), np.zeros(chains)
        caps = np.zeros(1, dtype=np.int32)
        t0 = time.perf_counter()
        ev = oracle.lib().or_evolve(pb.c, nt, w.seed_sampler, rep, chains, oracle._ptr(surv), oracle._ptr(surv_l),
                                    w.n_live - k, oracle._ptr(chol), lstar, steps_per_dim * d, 64, 64,
                                    oracle._ptr(new_u), oracle._ptr(new_l), oracle._ptr(caps))
        tot_s += time.perf_counter() - t0
        tot_ev += ev
        rep += 1
    return {"config": name, "form": "oracle", "evals_per_s": tot_ev / tot_s, "cores": nt,
            "sample": f"{rep} x {chains} chains of {steps_per_dim * d} slice steps from the first iteration "
                      f"({tot_ev} evaluations, {tot_s:.1f} s)"}


def run_table(args):
    """One JSON line per (workload, form): full runs of c0, c1, c2 and c4 on
    1024 coarse bins (FP64 and mixed), c4 on the full grid (mixed: the whole
    run; FP64: one iteration, and the batched likelihood), and the oracle's rate
    per workload."""
    import torch
    import paper_2509_24949_gb300 as g
    from paper_2509_24949_gb300 import _build
    if not _build.up_to_date():
        _build.build()
    stream = torch.cuda.Stream()
    rows = []
    for name in ("c0", "c1", "c2"):
        for prec in (g.NS_FP64, g.NS_MIXED):
            rows.append(table_row(g, name, prec, stream))
    for prec in (g.NS_FP64, g.NS_MIXED):
        rows.append(table_row(g, "c4", prec, stream, coarse=True))
    rows.append(table_row(g, "c4", g.NS_MIXED, stream))                  # the whole run (~17 s)
    rows.append(table_row(g, "c4", g.NS_FP64, stream, max_steps=1))      # one iteration (~9 s)
    for name in ("c2", "c4"):
        rows.append(batch_eval_row(g, name, g.NS_FP64, stream, points=2048))
        rows.append(batch_eval_row(g, name, g.NS_MIXED, stream, points=8192))
    if not args.no_oracle:
        for name, chains, spd in (("c0", 64, 5), ("c1", 64, 5), ("c2", 32, 2), ("c4", 16, 1)):
            rows.append(oracle_rate(name, chains, spd, 8.0))
    for r in rows:
        print(json.dumps(r), flush=True)


def run_scaling_study(args):
    """Runtime of whole runs against the live-point count (k = n/2) and against
    the deletion count k at n = 1000 (the paper's parallelism study, Sec. 4),
    on the 3-detector 4017-bin workload; one JSON line per run."""
    import torch
    import paper_2509_24949_gb300 as g
    from paper_2509_24949_gb300 import _build
    if not _build.up_to_date():
        _build.build()
    prec = g.NS_MIXED if args.precision == "mixed" else g.NS_FP64
    stream = torch.cuda.Stream()
    runs = [(n, n // 2) for n in (125, 250, 500, 1000, 2000, 4000)]
    runs += [(1000, k) for k in (10, 50, 100, 250, 750, 900)]
    for n, k in runs:
        w = gi.workload("c1")
        w.n_live, w.k = n, k
        sp, th = g.make_analysis(w, precision=prec, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it = sp.run()
        r = sp.result(samples=False)
        t1 = time.perf_counter()
        st = sp.stats()
        sp.close()
        print(json.dumps({"study": "runtime vs n and k", "workload": "c1", "precision": args.precision,
                          "n_live": n, "k": k, "iterations": it, "seconds": t1 - t0, "evals": st["evals"],
                          "evals_per_s": st["evals"] / (t1 - t0), "logZ": r["logZ"], "dlogZ": r["dlogZ"]}),
              flush=True)


def run_calibration(args):
    """Evidence calibration (paper Sec. 4 leaves its validation open): on the
    c1 workload, log Z over sampler seeds on the same data against the
    replicate error dlogZ, for 5, 10 and 20 slice steps per dimension; and the
    log Bayes factor of noise-only data against that of the SNR-20 injection."""
    import torch
    import paper_2509_24949_gb300 as g
    from paper_2509_24949_gb300 import _build
    if not _build.up_to_date():
        _build.build()
    prec = g.NS_MIXED if args.precision == "mixed" else g.NS_FP64
    stream = torch.cuda.Stream()
    seeds = 12
    for spd in (5, 10, 20):
        z, dz, secs = [], [], []
        for i in range(seeds):
            w = gi.workload("c1")
            w.steps_per_dim = spd
            w.seed_sampler += 1000 * (i + 1)
            sp, th = g.make_analysis(w, precision=prec, stream=stream.cuda_stream)
            t0 = time.perf_counter()
            sp.run()
            r = sp.result(samples=False)
            secs.append(time.perf_counter() - t0)
            sp.close()
            z.append(r["logZ"])
            dz.append(r["dlogZ"])
        z = np.array(z)
        print(json.dumps({"study": "log Z scatter over sampler seeds vs dlogZ", "workload": "c1",
                          "precision": args.precision, "steps_per_dim": spd, "seeds": seeds,
                          "mean_logZ": float(z.mean()), "sd_logZ": float(z.std(ddof=1)),
                          "mean_dlogZ": float(np.mean(dz)), "ratio_sd_to_dlogZ": float(z.std(ddof=1) / np.mean(dz)),
                          "mean_seconds": float(np.mean(secs))}), flush=True)
    # noise only: the same detectors and noise, no signal
    for label, snr_scale in (("noise only", 0.0), ("injection SNR 20", 1.0)):
        w = gi.workload("c1")
        probe, th = g.make_analysis(w, precision=g.NS_FP64, n_live=2, k=1, stream=stream.cuda_stream)
        data = snr_scale * probe.waveform(th)
        probe.close()
        data = data + gi.noise(w.seed_noise, np.tile(gi.psd_analytic(w.freqs()), (w.n_det, 1)), w.df)
        sp = g.sampler_for_workload(w, data=data, precision=prec, stream=stream.cuda_stream)
        sp.run()
        r = sp.result(samples=False)
        sp.close()
        print(json.dumps({"study": "log Bayes factor against noise", "workload": "c1", "data": label,
                          "precision": args.precision, "logZ": r["logZ"], "dlogZ": r["dlogZ"],
                          "rho2_over_2": float(probe_snr2(g, w, th, stream) / 2) if snr_scale else 0.0}),
              flush=True)


def run_population_calibration(args):
    """Evidence calibration over a population of injections (paper Sec. 4
    leaves the validation of its evidence estimates open): --injections
    synthetic 4017-bin analyses (3 detectors, 11 parameters; each its own
    injection drawn from the prior and scaled to SNR 20, and its own noise),
    each run with --seeds sampler seeds at 5, 10 and 20 slice steps per
    dimension. Per injection the runs' mean log Z stands in for the unknown
    true value; z = (log Z - mean) / (dlogZ sqrt(1 - 1/R)) is N(0, 1) if the
    reported dlogZ is the run-to-run error. One JSON line per chain length:
    the fractions of |z| < 1 and < 2 (0.68 and 0.95 if calibrated) and the
    pooled scatter over the mean reported dlogZ."""
    import torch
    import paper_2509_24949_gb300 as g
    from paper_2509_24949_gb300 import _build
    if not _build.up_to_date():
        _build.build()
    prec = g.NS_MIXED if args.precision == "mixed" else g.NS_FP64
    stream = torch.cuda.Stream()
    R = max(2, args.seeds)
    per_spd = {5: [], 10: [], 20: []}
    t0 = time.perf_counter()
    for i in range(args.injections):
        w = gi.workload("c1")
        w.seed_injection += 10 * (i + 1)
        w.seed_noise += 10 * (i + 1)
        inputs, th = workload_data(g, w, stream)
        for spd in per_spd:
            z, dz = [], []
            for r in range(R):
                sp = sampler_on(g, w, inputs, prec, stream, steps_per_dim=spd,
                                seed=w.seed_sampler + 7919 * (r + 1) + 104729 * i)
                sp.run()
                res = sp.result(samples=False)
                sp.close()
                z.append(res["logZ"])
                dz.append(res["dlogZ"])
            per_spd[spd].append((np.array(z), np.array(dz)))
    for spd, runs in per_spd.items():
        zs, ratio_num, ratio_den = [], [], []
        for z, dz in runs:
            dev = z - z.mean()
            zs.extend(dev / (dz * math.sqrt(1.0 - 1.0 / R)))
            ratio_num.append(np.var(z, ddof=1))
            ratio_den.append(np.mean(dz) ** 2)
        zs = np.abs(np.array(zs))
        print(json.dumps({"study": "evidence calibration over injections", "workload": "c1",
                          "precision": args.precision, "steps_per_dim": spd, "injections": len(runs),
                          "seeds_per_injection": R, "frac_within_1_dlogZ": float(np.mean(zs < 1.0)),
                          "frac_within_2_dlogZ": float(np.mean(zs < 2.0)),
                          "pooled_sd_over_mean_dlogZ": float(math.sqrt(np.mean(ratio_num) / np.mean(ratio_den))),
                          "mean_dlogZ": float(np.mean([np.mean(d) for _, d in runs])),
                          "seconds": time.perf_counter() - t0}), flush=True)


def probe_snr2(g, w, th, stream):
    sp = g.sampler_for_workload(w, data=None, precision=g.NS_FP64, n_live=2, k=1, stream=stream.cuda_stream)
    v = sp.snr2(th)
    sp.close()
    return v


def run_kernel_study(args):
    """Slice sampling against the random-walk (acceptance-walk) inner kernel on
    the c1 workload: time to log Z, evaluations and log Z over sampler seeds."""
    import torch
    import paper_2509_24949_gb300 as g
    from paper_2509_24949_gb300 import _build
    if not _build.up_to_date():
        _build.build()
    prec = g.NS_MIXED if args.precision == "mixed" else g.NS_FP64
    stream = torch.cuda.Stream()
    seeds = 8
    for kname, kern in (("slice", g.NS_KERNEL_SLICE), ("walk", g.NS_KERNEL_WALK)):
        z, dz, secs, evs, its = [], [], [], [], []
        for i in range(seeds):
            w = gi.workload("c1")
            w.seed_sampler += 1000 * (i + 1)
            sp, th = g.make_analysis(w, precision=prec, stream=stream.cuda_stream, kernel=kern)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it = sp.run()
            r = sp.result(samples=False)
            secs.append(time.perf_counter() - t0)
            evs.append(sp.stats()["evals"])
            its.append(it)
            sp.close()
            z.append(r["logZ"])
            dz.append(r["dlogZ"])
        z = np.array(z)
        print(json.dumps({"study": "inner kernel", "workload": "c1", "precision": args.precision,
                          "kernel": kname, "seeds": seeds, "mean_seconds": float(np.mean(secs)),
                          "mean_iterations": float(np.mean(its)), "mean_evals": float(np.mean(evs)),
                          "evals_per_s": float(np.sum(evs) / np.sum(secs)), "mean_logZ": float(z.mean()),
                          "sd_logZ": float(z.std(ddof=1)), "mean_dlogZ": float(np.mean(dz))}), flush=True)


def run_precision_study(args):
    """precision_agreement on one workload, one JSON line."""
    import torch
    import paper_2509_24949_gb300 as g
    from paper_2509_24949_gb300 import _build
    if not _build.up_to_date():
        _build.build()
    stream = torch.cuda.Stream()
    w = gi.workload(args.precision_study)
    r = precision_agreement(g, w, stream, seeds=args.seeds, name=args.precision_study)
    print(json.dumps({"study": "mixed against FP64", **r}), flush=True)


def run_profile_case(args):
    """A few iterations of one workload and form, untimed, for profiler captures
    of its kernels (e.g. ncu -k regex:k_slice -s <warm-up launches> -c 1)."""
    import torch
    import paper_2509_24949_gb300 as g
    from paper_2509_24949_gb300 import _build
    if not _build.up_to_date():
        _build.build()
    prec = g.NS_MIXED if args.precision == "mixed" else g.NS_FP64
    stream = torch.cuda.Stream()
    if args.batch_points:
        # the batched likelihood: ns_init's 8-point live set, one warm-up launch,
        # then `steps` launches of batch_points prior draws
        r = batch_eval_row(g, args.profile_case, prec, stream, points=args.batch_points, reps=args.steps)
        print(json.dumps({"profile_case": args.profile_case, "precision": args.precision, **r}))
        return
    w = gi.workload(args.profile_case)
    if args.n_live:
        w.n_live = args.n_live
    if args.k:
        w.k = args.k
    sp, th = g.make_analysis(w, precision=prec, stream=stream.cuda_stream)
    for _ in range(args.steps):
        sp.step()
    st = sp.stats()
    sp.close()
    print(json.dumps({"profile_case": args.profile_case, "precision": args.precision, "n_live": w.n_live,
                      "k": w.k, "iterations": st["iterations"], "evals": st["evals"],
                      "point_bins": st["point_bins"], "mixed_tile": st["mixed_tile"], "status": st["status"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gwns", choices=["gwns", "reference"])
    ap.add_argument("--core-only", action="store_true",
                    help="measure the timed steps and e2e only, without the time-to-logZ, serving, "
                         "agreement and CPU-baseline reports (for profiler runs); the timed region "
                         "is the same")
    ap.add_argument("--table", action="store_true",
                    help="per-workload table (full runs of c0-c2 and c4 on coarse bins, c4 full grid, "
                         "oracle rates): one JSON line each")
    ap.add_argument("--no-oracle", action="store_true", help="with --table: skip the oracle rates")
    ap.add_argument("--profile-case", default=None,
                    help="workload (c0..c4): run --steps untimed iterations for a profiler capture")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--kernel-study", action="store_true",
                    help="slice sampling vs the random-walk inner kernel on c1 (time, evaluations, log Z)")
    ap.add_argument("--calibration", action="store_true",
                    help="log Z scatter over seeds vs dlogZ (5, 10, 20 steps per dim) and noise-only log BF (c1)")
    ap.add_argument("--scaling-study", action="store_true",
                    help="whole-run time against n_live (k = n/2) and against k at n = 1000 (c1)")
    ap.add_argument("--precision-study", default=None,
                    help="mixed against FP64 on one workload (c0, c1, c2): per-point log L on 4096 prior "
                         "draws and log Z over --seeds sampler seeds")
    ap.add_argument("--seeds", type=int, default=8)
    ap.add_argument("--injections", type=int, default=0,
                    help="evidence calibration over this many injections (c1; --seeds runs each at 5, 10, "
                         "20 steps per dimension)")
    ap.add_argument("--n-live", type=int, default=0)
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--batch-points", type=int, default=0,
                    help="with --profile-case: time the batched likelihood on this many prior draws "
                         "(--steps launches) instead of running iterations")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.precision_study:
        run_precision_study(args)
        return
    if args.injections:
        run_population_calibration(args)
        return
    if args.table:
        run_table(args)
        return
    if args.profile_case:
        run_profile_case(args)
        return
    if args.scaling_study:
        run_scaling_study(args)
        return
    if args.calibration:
        run_calibration(args)
        return
    if args.kernel_study:
        run_kernel_study(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
