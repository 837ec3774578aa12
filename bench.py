"""Benchmark: likelihood evaluations per second inside nested-sampling
iterations on one GB300 (plus time-to-logZ, per-step latency and the mixed
precision form), on the 3-detector / 11-parameter / 4017-bin workload with
1000 live points and 500 chains per iteration.

A step is one ns_step: selection of the 500 lowest live points, evidence
update, survivors' covariance and Cholesky factor, 500 slice-sampling chains
of 55 steps each (every candidate's TaylorF2 likelihood on the GPU), and the
stopping test. Inputs are synthetic and seeded (gwinputs); the injection is
made with the library's own waveform.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (plain FP64 C, all host cores) on a
bounded sample of the same workload. Under torchrun each rank runs an
independent replica (different seeds); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gwinputs as gi  # noqa: E402

METRIC = "logL evals/sec (FP64, in nested-sampling iterations)"
UNIT = "evals/s"
WORKLOAD = "c1"
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
# FP64 pipe peak derived from the unit count: 2 FP64 FMA per clock per SM
# (1.25 TFLOP/s nominal over 152 SMs at 2070 MHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# Algorithmic FP64 work of one point-bin of the FP64 likelihood with D
# detectors, in FMA-equivalents: 8 basis FMAs + one sincos (32 FMA-equivalents
# on this GPU) + per detector 4 (phasor product) + 4 (complex MAC) + 4
# (phasor rotation). 1 FMA = 2 flops.
K_SLICE_FP64_C1_DRAM_BYTES = 547328   # ncu dram__bytes_read.sum + dram__bytes_write.sum of the current kernel


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


def build_workload(g, precision, seed_offset=0):
    w = gi.workload(WORKLOAD)
    w.seed_sampler += 100 * seed_offset
    w.seed_noise += 100 * seed_offset
    w.seed_injection += 100 * seed_offset
    return w


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
    w = build_workload(g, g.NS_FP64, rank)
    sp, th_inj = g.make_analysis(w, precision=g.NS_FP64, stream=stream.cuda_stream)
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush():
        with torch.cuda.stream(stream):
            l2_flush.fill_(1.0)

    for _ in range(args.warmup):
        sp.step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    st0 = sp.stats()
    evals0 = st0["evals"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for i in range(args.steps):
            flush()
            ev[i][0].record(stream)
            sp.step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    st1 = sp.stats()
    evals = st1["evals"] - evals0
    total_ms_max, evals_all = reduce_ranks(dist, total_ms, evals)
    value = evals_all / (total_ms_max / 1e3)

    roof = slice_kernel_roofline(st0, st1, args.steps, w.n_det)
    sp.close()

    # time-to-logZ, FP64 and mixed, full runs from ns_init to ns_result
    ttl = {}
    if not args.core_only:
        for name, prec in (("fp64", g.NS_FP64), ("mixed", g.NS_MIXED)):
            ttl[name] = time_to_logz(g, w, prec, stream)

    # end-to-end through the C ABI with host buffers: ns_init from host arrays,
    # then K ns_step_host calls that copy each iteration's dead points to host
    e2e = e2e_run(g, w, args.steps, stream)

    # the serving workload (64 analyses arriving at 2/s): p50/p99 time-to-logZ
    extras = rank == 0 and not args.core_only
    serving = serving_stream(g) if extras else None
    agreement = precision_agreement(g, w, stream) if extras else None
    # the mixed-precision likelihood against its roofline: the batched
    # likelihood on the 519,169-bin workload (8192 prior draws, three launches)
    mixed_lik = mixed_likelihood_roofline(g, stream) if extras else None

    if rank == 0:
        cpu = cpu_baseline() if ws == 1 and not args.core_only else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded noise, TaylorF2 injection at SNR 20, seeded detectors)",
            "config": {"workload": "c1: 3 detectors, 11 parameters, 20-1024 Hz at df=0.25 (4017 bins), "
                                   "n_live=1000, k=500, 55 slice steps per chain, FP64",
                       "parallelism": f"replicas{ws}", "l2": "flushed before every timed step (256 MB write)"},
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "time_to_logZ": ttl,
            "serving": serving,
            "mixed_vs_fp64": agreement,
            "mixed_likelihood": mixed_lik,
            "e2e": e2e,
            "gpu_launches": 5 * args.steps,   # the 5 library kernels of each ns_step (the L2 flush fill is torch's)
            "kernel_ms_per_step": [(b - a) / args.steps for a, b in zip(st0["kernel_ms"], st1["kernel_ms"])],
            "roofline": roof,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def mixed_likelihood_roofline(g, stream):
    """The mixed batched likelihood (`ns_eval_lnl`, kernel k_eval) on the c4
    grid: throughput and the fraction of its binding pipe (derived peaks, as
    for the mixed rows of the table)."""
    r = batch_eval_row(g, "c4", g.NS_MIXED, stream, points=8192, reps=3)
    peak = FP32_LANE_OPS if r["pipe"] == "FP32" else SFU_LANE_OPS
    return {"workload": "c4: 3 detectors, 20-2048 Hz at df=1/256 (519,169 bins), 8192 prior draws, "
                        "mixed precision, 128-bin tiles", "kernel": "k_eval<MIXED,3 det>",
            "evals_per_s": r["batch_evals_per_s"], "point_bins_per_s": r["point_bins_per_s"],
            "bound": r["pipe"], "frac": r["frac"], "peak_lane_ops_per_s": peak,
            "instr_per_point_bin": (mixed_fp32_per_point_bin(3, r["mixed_tile"]) if r["pipe"] == "FP32"
                                    else mixed_mufu_per_point_bin(3, r["mixed_tile"])),
            "peak_source": "derived (not measured): 128 FP32 / 16 MUFU lanes/clk/SM x 152 SMs x 2070 MHz"}


def slice_kernel_roofline(st0, st1, steps, n_det):
    """Roofline of the fused slice-update kernel over the timed region: its
    average launch duration from the CUDA events recorded around it inside the
    iteration's graph (on the library's stream), and its algorithmic FP64 work
    = point-bins processed (device-side count of jcut+1 per evaluation) x the
    FMA-equivalents of one point-bin."""
    ms = (st1["kernel_ms"][3] - st0["kernel_ms"][3]) / steps
    pb = (st1["point_bins"] - st0["point_bins"]) / steps
    ev = (st1["evals"] - st0["evals"]) / steps
    flops = pb * fp64_flops_per_point_bin(n_det)
    achieved = flops / (ms / 1e3) / 1e12 if ms > 0 else None
    share = ms / (sum(st1["kernel_ms"]) - sum(st0["kernel_ms"])) * steps if ms > 0 else None
    return {"bound": "alu", "kernel": "k_slice<FP64,3 det> (fused slice update + likelihood)",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
            # dram__bytes_read.sum + dram__bytes_write.sum of one k_slice<FP64> launch on this
            # workload (profiles/k_slice_fp64_c1_ncu_full.md); null once the kernel changes
            "traffic": K_SLICE_FP64_C1_DRAM_BYTES,
            "peak_source": "derived (not measured): 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz",
            "per_launch": {"ms": ms, "evals": ev, "point_bins": pb,
                           "flops_per_point_bin": fp64_flops_per_point_bin(n_det),
                           "share_of_step_kernels": share}}


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


def precision_agreement(g, w, stream, seeds: int = 16, points: int = 4096, name: str = WORKLOAD):
    """Mixed against FP64 on the GPU: per-point log L difference on prior
    draws, and log Z over `seeds` sampler seeds (same data), reported as the
    mean difference with its standard error."""
    sp64, th = g.make_analysis(w, precision=g.NS_FP64, stream=stream.cuda_stream)
    spmx, _ = g.make_analysis(w, precision=g.NS_MIXED, stream=stream.cuda_stream)
    u = gi.unit_cube(777, points, w.dim)
    d = np.abs(spmx.eval_lnl(u) - sp64.eval_lnl(u))
    sp64.close()
    spmx.close()
    dz, z64 = [], []
    for i in range(seeds):
        zs = []
        for prec in (g.NS_FP64, g.NS_MIXED):
            w2 = gi.workload(name)
            w2.seed_sampler += 1000 * (i + 1)
            sp, _ = g.make_analysis(w2, precision=prec, stream=stream.cuda_stream)
            sp.run()
            zs.append(sp.result(samples=False)["logZ"])
            sp.close()
        dz.append(zs[1] - zs[0])
        z64.append(zs[0])
    dz = np.array(dz)
    return {"workload": name, "points": points, "max_abs_dlogL": float(d.max()),
            "rms_dlogL": float(np.sqrt(np.mean(d * d))),
            "seeds": seeds, "mean_dlogZ": float(dz.mean()), "stderr_dlogZ": float(dz.std(ddof=1) / np.sqrt(seeds)),
            "max_abs_dlogZ_single_seed": float(np.abs(dz).max()), "sd_logZ_fp64_over_seeds": float(np.std(z64, ddof=1))}


def e2e_run(g, w, steps, stream):
    import torch
    probe, th = g.make_analysis(w, precision=g.NS_FP64, stream=stream.cuda_stream)
    # host inputs of the analysis (pinned copies not needed: the ABI copies them)
    f = w.freqs()
    psd = np.tile(gi.psd_analytic(f), (w.n_det, 1))
    data = probe.waveform(th) + gi.noise(w.seed_noise, psd, w.df)
    probe.close()
    pos, xarm, yarm = gi.detectors(w.seed_geometry, w.n_det)
    k, d = w.k, w.dim
    du, dl, dw = np.zeros((k, d)), np.zeros(k), np.zeros(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sp = g.Sampler(kind=w.kind, lo=w.lo, hi=w.hi, data=data, psd=psd, f0=w.f0, df=w.df, pos=pos,
                   xarm=xarm, yarm=yarm, n_live=w.n_live, k=k, steps_per_dim=w.steps_per_dim,
                   precision=g.NS_FP64, seed=w.seed_sampler, stream=stream.cuda_stream)
    for _ in range(steps):
        sp.step_host(k, du, dl, dw)
    t1 = time.perf_counter()
    ev = sp.stats()["evals"]
    sp.close()
    h2d = (2 * data.size + psd.size) * 8
    return {"value": ev / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": k * (d + 2) * 8,
            "note": "ns_init from host arrays (data, PSD upload amortised over the steps) + ns_step_host"}


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


def oracle_sample(chains: int, iteration: int = 0):
    """One bounded sample of the workload on the oracle: from the initial live
    set, the first iteration's selection and covariance, then `chains` of its
    500 slice-sampling chains (iteration index `iteration` keys the draws)."""
    import oracle
    from oracle import ns as ons
    w = gi.workload(WORKLOAD)
    if not hasattr(oracle_sample, "cache"):
        pb, th = oracle.make_problem(w)
        st0 = ons.initial_state(pb, w.n_live, w.seed_sampler)
        oracle_sample.cache = (pb, st0)
    pb, st0 = oracle_sample.cache
    d = pb.dim
    order = np.argsort(st0.live_logl, kind="stable")
    k = w.k
    surv = np.ascontiguousarray(st0.live_u[order[k:]])
    surv_l = np.ascontiguousarray(st0.live_logl[order[k:]])
    chol = np.ascontiguousarray(ons.survivor_cholesky(surv))
    lstar = float(st0.live_logl[order[k - 1]])
    new_u = np.zeros((chains, d))
    new_l = np.zeros(chains)
    caps = np.zeros(1, dtype=np.int32)
    nt = oracle.max_threads()
    t0 = time.perf_counter()
    ev = oracle.lib().or_evolve(pb.c, nt, w.seed_sampler, iteration, chains, oracle._ptr(surv),
                                oracle._ptr(surv_l), w.n_live - k, oracle._ptr(chol), lstar,
                                w.steps_per_dim * d, 64, 64, oracle._ptr(new_u), oracle._ptr(new_l),
                                oracle._ptr(caps))
    return ev, time.perf_counter() - t0, nt


def cpu_baseline(target_s: float = 10.0):
    """The oracle's chain work of whole iterations (500 chains each) until
    about target_s seconds of wall time on all host cores."""
    tot_ev, tot_s, reps, nt = 0, 0.0, 0, 1
    while tot_s < target_s and reps < 200:
        ev, sec, nt = oracle_sample(500, iteration=reps)
        tot_ev += ev
        tot_s += sec
        reps += 1
    return {"value": tot_ev / tot_s, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"{reps} x the 500 slice-sampling chains of the first iteration of c1 "
                      f"({tot_ev} evaluations, {tot_s:.1f} s), plain FP64 C, OpenMP over chains"}


def run_reference(args):
    """The oracle as the reference arm: each step evolves the 500 chains of one
    iteration (from the initial live set, draws keyed by the step index)."""
    ws, rank = world()
    if rank != 0:
        return
    for i in range(args.warmup):
        oracle_sample(500, iteration=1000 + i)
    tot_ev, tot_s, nt = 0, 0.0, 1
    for i in range(args.steps):
        ev, sec, nt = oracle_sample(500, iteration=i)
        tot_ev += ev
        tot_s += sec
    value = tot_ev / tot_s
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": "c1: 3 detectors, 11 parameters, 20-1024 Hz at "
                                                      "df=0.25 (4017 bins), n_live=1000, k=500, 55 slice "
                                                      "steps per chain, FP64"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                            "sample": "per step: the 500 chains of one iteration from the initial live set"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


FP32_LANE_OPS = 152 * 128 * 2.070e9    # FP32 pipe: 128 lanes/clk/SM x 152 SMs x 2070 MHz
SFU_LANE_OPS = 152 * 16 * 2.070e9      # MUFU (sin, cos): 16 lanes/clk/SM x 152 SMs x 2070 MHz


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
    return {"config": name + (" (1024 coarse bins)" if coarse else ""),
            "form": "fp64" if precision == g.NS_FP64 else "mixed", "iterations": it, "done": done,
            "evals": ev, "evals_per_s": ev / (sum(ms) / 1e3), "point_bins_per_s": pb / (sum(ms) / 1e3),
            "bins_per_eval": pb / max(ev, 1), "k_slice_frac": frac, "k_slice_pipe": pipe,
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
           "warps_per_point": warps or None,
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
    1024 coarse bins (FP64 and mixed), c4 on the full grid (mixed: 2 iterations;
    FP64: batched likelihood), and the oracle's rate per workload."""
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
    rows.append(table_row(g, "c4", g.NS_MIXED, stream, max_steps=2))
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
