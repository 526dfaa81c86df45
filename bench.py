#!/usr/bin/env python
"""Benchmark: joint FFT-BP decoded frames/s on GB300.

Workload (one step = one batch through the whole decoder): K = 4 users, GF(16)
regular (2,4) LDPC code with n = 256 symbols, PAM-sum AWGN channel, 65,536 frames
per batch, at most 50 iterations with per-frame syndrome early stop; the SNR
sweep 6, 8, ..., 16 dB is covered by cycling one SNR per step.  Inputs are seeded
synthetic frames (uniform information symbols, random-permutation code with
4-cycles removed, uniform nonzero coefficients).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  For N > 1 launch under torch.distributed.run:
every rank decodes its own batch (independent frames, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "joint-BP decoded frames/s at matched SER vs plain form; served p50/p99 latency"
K_USERS, Q, N_SYM, FRAMES, ITERS = 4, 16, 256, 65536, 50
SNRS = [6.0, 8.0, 10.0, 12.0, 14.0, 16.0]
WORKLOAD = ("K=4 users, GF(16) regular (2,4) LDPC, n=256, PAM-sum AWGN, 65,536 frames per batch, "
            "SNR 6-16 dB in 2 dB steps (one SNR per step), 50 iterations with syndrome early stop")


def frame_seed(snr_idx: int, rank: int) -> int:
    return 2 * 10**9 + snr_idx * 10**6 + rank


def make_inputs(rank: int, F: int):
    from paper_2605_26580_gb300 import inputs as I
    code = I.make_code(N_SYM, Q)
    base = I.make_frames(code, K_USERS, SNRS[0], F, seed=frame_seed(0, rank))
    ys, sig = [], []
    for i, snr in enumerate(SNRS):
        y, s2 = I.channel_output(Q, base["c"], base["perm"], snr, frame_seed(i, rank) + 1)
        ys.append(y)
        sig.append(s2)
    return code, base, ys, sig


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- algorithmic counts

def channel_macs_per_use(K: int, q: int) -> int:
    """Multiply-adds of the channel node per channel use.  K <= 4 (q <= 16): the
    split-user scheme (K = 2: two correlations with G; K = 3: prefix mu_0*mu_1,
    two correlations with G, two with the suffix; K = 4: for each half a pair
    convolution, a correlation with G and two output correlations).  Otherwise the
    prefix/suffix chain: prefixes F_2..F_{K-1}, suffixes B_{K-1}..B_1, K-1 outputs."""
    D = q - 1
    if K == 1:
        return 0
    if K == 2 and q <= 16:
        return 2 * q * q
    if K == 3 and q <= 16:
        return q * q + 2 * q * (2 * D + 1) + 2 * q * q
    if K == 4 and q <= 16:
        return 2 * (q * q + (2 * D + 1) ** 2 + 2 * q * q)
    fwd = sum((j * D + 1) * q for j in range(1, K - 1))
    bwd = sum((k * D + 1) * q for k in range(1, K))
    out = sum((k * D + 1) * q for k in range(1, K))
    return fwd + bwd + out


def flops_per_frame_iter(K: int, q: int, n: int, dc: int = 4) -> float:
    """Algorithmic FP32 operations of one iteration of one frame (the roofline's
    count): 2 per channel multiply-add; per check and user 2 dc transforms of
    q log2 q additions and 6 q leave-one-out products; per variable and user 5 q
    products (message into the channel node, the two v2c, the posterior)."""
    P = n * 2 // dc
    chan = 2.0 * channel_macs_per_use(K, q) * n
    check = K * P * (2 * dc * q * math.log2(q) + 6 * q)
    var = K * n * q * 5
    return chan + check + var


def fp32_peak_tflops(sm_count: int, clock_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return sm_count * 128 * 2 * clock_mhz * 1e6 / 1e12


def measured_fp32_peak(jbp, device: int, seconds: float = 1.5) -> dict:
    """The device's FP32 multiply-add rate, measured now (jbp_fp32_peak) with
    scalar FFMA and with two-lane FFMA2 instructions, clocks sampled meanwhile;
    the peak is the larger rate."""
    clocks = ClockSampler(device)
    clocks.start()
    time.sleep(0.2)
    ffma = jbp.fp32_peak(device, seconds, packed=False)
    ffma2 = jbp.fp32_peak(device, seconds, packed=True)
    clk = clocks.stop()
    return {"tflops": max(ffma, ffma2), "ffma": ffma, "ffma2": ffma2, "seconds": seconds, "clocks": clk}


def hbm_peak_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def aggregate(local_ms: float, local_frames: int, dist=None, device=None):
    """Whole-job throughput over replicas: every rank decodes its own frames (no
    data exchange); the job time is the max over ranks.  Returns (max_ms, frames/s)."""
    world = 1
    total_ms = local_ms
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * local_frames / (total_ms / 1e3)


# --------------------------------------------------------------------------- reference arm (the oracle)

def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    from paper_2605_26580_gb300 import inputs as I
    S = args.ref_frames or max(4, os.cpu_count() or 1)
    cores = min(os.cpu_count() or 1, S)      # the oracle spreads frames over threads
    code = I.make_code(N_SYM, Q)
    base = I.make_frames(code, K_USERS, SNRS[0], S, seed=frame_seed(0, 0))
    samples = []
    for i, snr in enumerate(SNRS):
        y, s2 = I.channel_output(Q, base["c"], base["perm"], snr, frame_seed(i, 0) + 1)
        samples.append((y, s2))
    times = []
    for s in range(args.warmup + args.steps):
        y, s2 = samples[s % len(SNRS)]
        t0 = time.perf_counter()
        O.decode(code, K_USERS, s2, base["perm"], y, ITERS, early_stop=True, threads=cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = S * len(times) / total
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "K": K_USERS, "q": Q, "n": N_SYM, "iters": ITERS, "snr_db": SNRS,
                   "frames_per_step": S},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": "%d frames of the workload per step (the full batch is 65,536), FP64 "
                                   "oracle, OpenMP over frames on %d host threads" % (S, cores)},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_leg() -> dict:
    from oracle import oracle as O
    O.build()
    from paper_2605_26580_gb300 import inputs as I
    cores = os.cpu_count() or 1
    # about 10-20 s of CPU work on the host's cores (one frame is ~1.1 s of one core)
    S = max(16, 12 * cores)
    code = I.make_code(N_SYM, Q)
    fr = I.make_frames(code, K_USERS, 10.0, S, seed=frame_seed(2, 0))
    t0 = time.perf_counter()
    O.decode(code, K_USERS, fr["sigma2"], fr["perm"], fr["y"], ITERS, early_stop=True, threads=cores)
    dt = time.perf_counter() - t0
    # the same oracle on one core, on the first 8 of those frames (about 9 s)
    S1 = 8
    t0 = time.perf_counter()
    O.decode(code, K_USERS, fr["sigma2"], fr["perm"], fr["y"][:S1], ITERS, early_stop=True, threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": S / dt, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": "%d frames at 10 dB of the same workload, FP64 oracle, %d threads, %.1f s" % (S, cores, dt),
            "one_core": {"value": S1 / dt1, "unit": "frames/s",
                         "sample": "first %d of those frames, 1 thread, %.1f s" % (S1, dt1)}}


# --------------------------------------------------------------------------- our arm

def make_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="fused", choices=["fused", "step", "auto"])
    ap.add_argument("--frames", type=int, default=FRAMES)
    ap.add_argument("--ref-frames", type=int, default=0)
    ap.add_argument("--no-extras", action="store_true", help="skip the plain/step/e2e/cpu legs")
    ap.add_argument("--snrs", type=int, default=len(SNRS), help="use only the first N SNR points")
    ap.add_argument("--config", default="headline",
                    choices=["headline", "small", "precision", "uneven", "serve", "ura"],
                    help="headline: the contract line (K=4, GF(16), n=256); the others print one JSON line "
                         "for the other workloads")
    ap.add_argument("--frac", type=float, default=1.0, help="fraction of the uneven/serving workload (tests)")
    ap.add_argument("--launch", default="auto", help="fused launch shape: auto (autotune), default, or THREADS,FPC")
    ap.add_argument("--variants", default="0,d0,3,1,2",
                    help="precision workload: check-node variants to run (dP: with the DFT channel node)")
    ap.add_argument("--channel-legs", type=int, default=1, help="precision workload: time the channel node alone")
    ap.add_argument("--channel-node", default="trellis", choices=["trellis", "dft", "auto"],
                    help="uneven and serving workloads: channel node (dft: tensor-core variant wherever it "
                         "applies; auto: except where the register-resident trellis applies)")
    ap.add_argument("--channel-frames", type=int, default=4096, help="precision workload: frames of that leg")
    ap.add_argument("--oracle-sample", type=int, default=16, help="precision workload: oracle frames")
    ap.add_argument("--block-iters", type=int, default=0,
                    help="serving: iterations per pool block (0 = the library's default)")
    ap.add_argument("--rates", default="250,500,1000,20000,50000,100000,200000",
                    help="serving workload: Poisson arrival rates (requests/s)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="headline: skip the other workloads' summary (small, precision, uneven, serving)")
    return ap


def main() -> None:
    args = make_parser().parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config != "headline":
        run_workload(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_26580_gb300 import jbp

    F = args.frames
    code, base, ys, sig = make_inputs(rank, F)
    ys, sig = ys[:args.snrs], sig[:args.snrs]
    ctx = jbp.Context(iters=ITERS, early_stop=True, precision=jbp.PREC_FP32, device=local)
    decs = [jbp.Decoder(ctx, code, K_USERS, s2, base["perm"]) for s2 in sig]
    form = {"fused": jbp.FORM_FUSED, "step": jbp.FORM_STEP, "auto": jbp.FORM_AUTO}[args.form]

    y_d = [torch.from_numpy(y).to(dev) for y in ys]                       # 6 x 67 MB > L2
    hat_d = [torch.empty((F, K_USERS, N_SYM), dtype=torch.uint8, device=dev) for _ in ys]
    it_d = [torch.empty((F,), dtype=torch.int32, device=dev) for _ in ys]
    ok_d = [torch.empty((F, K_USERS), dtype=torch.uint8, device=dev) for _ in ys]
    stream = torch.cuda.Stream(device=dev)

    def step(s):
        i = s % len(ys)
        decs[i].decode_device(y_d[i], hat_d[i], it_d[i], ok_d[i], form=form, stream=stream)

    launch = {"mode": args.launch}
    if args.launch == "auto":
        # one autotune (on the first SNR point's batch); every decoder uses that shape
        th, fc = decs[0].tune(y_d[0], hat_d[0], it_d[0], ok_d[0], stream=stream)
        for d in decs[1:]:
            d.set_launch(th, fc)
        launch.update(threads=th, frames_per_cta=fc, applies_to="all %d decoders" % len(decs))
    elif args.launch != "default":
        th, fc = (int(v) for v in args.launch.split(","))
        for d in decs:
            d.set_launch(th, fc)
        launch.update(threads=th, frames_per_cta=fc)
    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t_wall = time.perf_counter()
    for s in range(args.steps):
        starts[s].record(stream)
        step(args.warmup + s)
        ends[s].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms, value = aggregate(sum(step_ms), F * args.steps, dist, dev)

    # decisions of every SNR point (outside the timed region)
    ser, iters_mean = {}, {}
    for s in range(args.warmup, args.warmup + args.steps):
        i = s % len(ys)
        h = hat_d[i].cpu().numpy()
        ser[str(SNRS[i])] = float((h != base["c"]).mean())
        iters_mean[str(SNRS[i])] = float(it_d[i].float().mean().item())
    info_rate = value * K_USERS * code["k"]
    fallbacks = sum(d.log_fallbacks() for d in decs)

    # roofline of the dominant kernel: the fused decode kernel is the only launch
    # of a step, so its duration is the step's CUDA-event time
    it_total = sum(float(it_d[s % len(ys)].double().sum().item())
                   for s in range(args.warmup, args.warmup + args.steps))
    flops = flops_per_frame_iter(K_USERS, Q, N_SYM) * it_total
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_meas = measured_fp32_peak(jbp, local)
    peak = peak_meas["tflops"]
    achieved = flops / (total_ms / 1e3) / 1e12 / world
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                # DRAM bytes per 65,536-frame launch: ncu capture of k_fused_pos<16,4> in its lane-pair
                # shape (the autotuner's choice) on 1,216 frames (1.349 MB read + 14.1 KB written),
                # scaled by frames; state stays in shared memory, so this is y in (and decisions out
                # through L2), not message traffic.  Only valid at the default workload size and for
                # this kernel version.
                "traffic": (1.3635e6 * 65536 / 1216) if args.frames == FRAMES else None,
                "traffic_note": "per launch, from profiles/k_fused_pos_q16_k4_n256_small_full.md scaled by frames",
                "kernel": "k_fused_pos<16,4>",
                "peak_note": ("of measured: FP32 multiply-add peak measured in this run by jbp_fp32_peak "
                              "(independent FMA chains on all %d SMs, median of 3 launches, %.1f s; "
                              "FFMA %.2f, two-lane FFMA2 %.2f TFLOP/s; the larger is the peak) at a median "
                              "SM clock of %s MHz; derived nominal at that clock: %.2f TFLOP/s"
                              % (sm_count, peak_meas["seconds"], peak_meas["ffma"], peak_meas["ffma2"],
                                 peak_meas["clocks"].get("sm_mhz"),
                                 fp32_peak_tflops(sm_count, peak_meas["clocks"].get("sm_mhz") or 2070.0))),
                "peak_clocks": peak_meas["clocks"],
                "flops_per_frame_iter": flops_per_frame_iter(K_USERS, Q, N_SYM)}

    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "K": K_USERS, "q": Q, "n": N_SYM, "frames_per_batch": F,
                   "iters": ITERS, "early_stop": True, "snr_db": SNRS, "form": args.form,
                   "l2": "inputs cycle through 6 batches x %.0f MB (> 129 MB L2); message state in shared memory"
                         % (F * N_SYM * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single", "launch": launch},
        "info_symbols_per_s": info_rate,
        "ser": ser, "iters_mean": iters_mean,
        "log_fallbacks_per_channel_message": fallbacks / max(1.0, (args.warmup + args.steps) * F * N_SYM * K_USERS
                                                               * float(np.mean(list(iters_mean.values())))),
        "clocks": clk, "roofline": roofline,
        "gpu_launches": args.steps,
        "wall_s_timed": t_wall,
    }

    if rank == 0 and world == 1 and not args.no_extras:
        line.update(extra_legs(jbp, torch, dev, code, base, ys, sig, decs, stream))
        line["cpu_baseline"] = cpu_baseline_leg()
    for d in decs:
        d.close()
    ctx.close()
    if rank == 0 and world == 1 and not args.no_extras and not args.no_workloads:
        del y_d, hat_d, it_d, ok_d
        torch.cuda.empty_cache()
        line["workloads"] = other_workloads()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def other_workloads() -> dict:
    """The other workloads, each on a bounded sample stated in its key and its
    config, so that the default run stays within a few minutes: the small
    workload in full; the precision workload (K=4, GF(64), n=512) on a quarter of
    its 32,768 frames with an 8-frame oracle sample; the uneven batch on a tenth
    of its 100,000 frames; serving at two rates below the knee and one above it.
    A workload that fails is reported with its error instead of a result."""
    base = vars(make_parser().parse_args([]))
    runs = [
        ("small_K2_gf4_n64_1000_frames", wl_small, {}),
        ("precision_K4_gf64_n512_quarter_8192_frames", wl_precision,
         {"frac": 0.25, "oracle_sample": 2, "channel_legs": 0, "steps": 1}),
        ("uneven_tenth_10000_frames_auto_channel_node", wl_uneven, {"frac": 0.1, "channel_node": "auto", "steps": 1}),
        ("serving_4000_request_pool_auto_channel_node", wl_serve,
         {"frac": 0.2, "channel_node": "auto", "rates": "250,1000,20000"}),
    ]
    out = {}
    for key, fn, over in runs:
        a = argparse.Namespace(**{**base, **over})
        t0 = time.perf_counter()
        try:
            r = fn(a)
            r.pop("metric", None)
            r["wall_s"] = time.perf_counter() - t0
            out[key] = r
        except Exception as e:   # report, do not lose the headline line
            out[key] = {"error": "%s: %s" % (type(e).__name__, e), "wall_s": time.perf_counter() - t0}
    return out


def extra_legs(jbp, torch, dev, code, base, ys, sig, decs, stream) -> dict:
    """e2e through host buffers, the plain per-frame form, and the HBM step form."""
    F = ys[0].shape[0]
    out = {}
    # e2e: host (pinned) buffers through jbp_decode, copies inside the timed region
    i = min(2, len(ys) - 1)
    y_h = torch.from_numpy(ys[i]).pin_memory().numpy()
    times = []
    for r in range(3):
        t0 = time.perf_counter()
        res = decs[i].decode(y_h, form=jbp.FORM_AUTO)
        times.append(time.perf_counter() - t0)
    e2e = F / float(np.median(times))
    out["e2e"] = {"value": e2e, "unit": "frames/s", "h2d_bytes_per_step": F * N_SYM * 4,
                  "d2h_bytes_per_step": F * K_USERS * N_SYM + F * 4 + F * K_USERS,
                  "ser": float((res["hat"] != base["c"]).mean())}
    # plain per-frame form (one frame per launch sequence) on a sample
    S = 64
    t0 = time.perf_counter()
    pl = decs[i].decode(ys[i][:S], form=jbp.FORM_PLAIN)
    dt = time.perf_counter() - t0
    out["plain_form"] = {"value": S / dt, "unit": "frames/s", "sample": "%d frames at %.0f dB" % (S, SNRS[i]),
                         "ser": float((pl["hat"] != base["c"][:S]).mean()),
                         "matches_batched": bool(np.array_equal(pl["hat"], res["hat"][:S]))}
    # HBM step form on the full batch, with per-kernel events for the message-passing kernels
    y_d = torch.from_numpy(ys[i]).to(dev)
    hat = torch.empty((F, K_USERS, N_SYM), dtype=torch.uint8, device=dev)
    it = torch.empty((F,), dtype=torch.int32, device=dev)
    ok = torch.empty((F, K_USERS), dtype=torch.uint8, device=dev)
    decs[i].decode_device(y_d, hat, it, ok, form=jbp.FORM_STEP, stream=stream)   # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    decs[i].decode_device(y_d, hat, it, ok, form=jbp.FORM_STEP, stream=stream)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    sh = hat.cpu().numpy()
    # the fused form sums in another order; frames whose BP does not converge (all of
    # them past capacity) can end in different decisions, at equal symbol error rate
    out["step_form"] = {"value": F / (ms / 1e3), "unit": "frames/s",
                        "matches_fused": bool(np.array_equal(sh, res["hat"])),
                        "decisions_differing_from_fused": int((sh != res["hat"]).sum()),
                        "decisions": int(sh.size), "ser": float((sh != base["c"]).mean())}
    # single-step kernels on the full batch: achieved HBM bandwidth vs algorithmic bytes
    E, n, q, K = code["P"] * code["dc"], N_SYM, Q, K_USERS
    msg = torch.ones((F, K, E, q), dtype=torch.float32, device=dev)
    ch2v = torch.empty((F, K, n, q), dtype=torch.float32, device=dev)
    post = torch.empty_like(ch2v)
    hbm = hbm_peak_gbs()
    kernels = {}
    msg_b, ch_b = F * K * E * q * 4, F * K * n * q * 4
    legs = [
        ("channel", lambda: decs[i].step_channel(y_d, msg, ch2v, stream=stream), msg_b + ch_b + msg_b + F * n * 4),
        ("check", lambda: decs[i].step_check(msg, stream=stream), 2 * msg_b),
        ("var", lambda: decs[i].step_var(ch2v, msg, None, hat, stream=stream), ch_b + msg_b + F * K * n),
    ]
    for name, fn, nbytes in legs:
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            fn()
        b.record(stream)
        stream.synchronize()
        t = a.elapsed_time(b) / 3 / 1e3
        kernels[name] = {"ms": t * 1e3, "algorithmic_bytes": nbytes, "gbs": nbytes / t / 1e9,
                         "frac_hbm": nbytes / t / 1e9 / hbm}
    out["hbm_step_kernels"] = kernels
    return out


# --------------------------------------------------------------------------- other workloads

def _ctx_dev():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_26580_gb300 import jbp
    torch.cuda.set_device(0)
    return jbp, torch, torch.device("cuda", 0)


def _timed(torch, stream, fn, steps):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) / 1e3 / steps


def run_workload(args):
    fn = {"small": wl_small, "precision": wl_precision, "uneven": wl_uneven, "serve": wl_serve,
          "ura": wl_ura}[args.config]
    line = fn(args)
    print(json.dumps(line), flush=True)


def wl_small(args):
    """K=2 users, GF(4), n=64, SNR 10 dB, 20 flooding iterations (no early stop),
    1,000 frames: FP32 GPU (fused) vs the FP64 oracle on all frames."""
    jbp, torch, dev = _ctx_dev()
    from oracle import oracle as O
    from paper_2605_26580_gb300 import inputs as I
    code = I.make_code(64, 4)
    F = 1000
    fr = I.make_frames(code, 2, 10.0, F, seed=1_000_000_000)
    ctx = jbp.Context(iters=20, early_stop=False)
    dec = jbp.Decoder(ctx, code, 2, fr["sigma2"], fr["perm"])
    y = torch.from_numpy(fr["y"]).to(dev)
    hat = torch.empty((F, 2, 64), dtype=torch.uint8, device=dev)
    it = torch.empty((F,), dtype=torch.int32, device=dev)
    ok = torch.empty((F, 2), dtype=torch.uint8, device=dev)
    st = torch.cuda.Stream()
    for _ in range(3):
        dec.decode_device(y, hat, it, ok, stream=st)
    sec = _timed(torch, st, lambda: dec.decode_device(y, hat, it, ok, stream=st), max(3, args.steps))
    t0 = time.perf_counter()
    host = dec.decode(fr["y"])
    e2e = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = O.decode(code, 2, fr["sigma2"], fr["perm"], fr["y"], 20, early_stop=False, want_margin=True, threads=cores)
    t_or = time.perf_counter() - t0
    g = hat.cpu().numpy()
    sure = ref["margin"] > 1e-6
    dec.close()
    ctx.close()
    return {"metric": METRIC, "value": F / sec, "unit": "frames/s", "config": {
                "workload": "K=2 users, GF(4) regular (2,4) LDPC, n=64, SNR 10 dB, 20 flooding iterations, "
                            "1,000 frames", "form": "fused"},
            "dtype": "f32", "ms_per_batch": sec * 1e3, "e2e_frames_per_s": F / e2e,
            "ser_gpu": float((g != fr["c"]).mean()), "ser_oracle": float((ref["hat"] != fr["c"]).mean()),
            "decisions_differing_at_margin_gt_1e-6": int(((g != ref["hat"]) & sure).sum()),
            "decisions_compared": int(sure.sum()),
            "cpu_baseline": {"value": F / t_or, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": "all 1,000 frames, 20 iterations"}}


def wl_precision(args):
    """K=4, GF(64), n=512, SNR 14 dB, 50 iterations (early stop), 32,768 frames:
    check node as FP32 butterflies vs tensor-core BF16X3 / BF16X2 (hi/lo) / BF16."""
    jbp, torch, dev = _ctx_dev()
    from oracle import oracle as O
    from paper_2605_26580_gb300 import inputs as I
    K, q, n, F = 4, 64, 512, int(32768 * args.frac)
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 14.0, F, seed=3_000_000_000, device=dev)
    y = torch.from_numpy(fr["y"]).to(dev)
    hat = torch.empty((F, K, n), dtype=torch.uint8, device=dev)
    it = torch.empty((F,), dtype=torch.int32, device=dev)
    ok = torch.empty((F, K), dtype=torch.uint8, device=dev)
    st = torch.cuda.Stream()
    S = args.oracle_sample
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = O.decode(code, K, fr["sigma2"], fr["perm"], fr["y"][:S], 50, early_stop=True, want_margin=True,
                   threads=cores) if S > 0 else None
    t_or = time.perf_counter() - t0
    rng = np.random.default_rng(7)
    E = code["P"] * 4
    v2c = np.exp(I.random_log_messages(rng, (8, K, E), q, spread=3.0)).astype(np.float32)
    c2v_o = O.step_check_v2c(code, K, np.log(v2c.astype(np.float64)))
    variants = {}
    names = {0: "fp32_butterfly", 3: "bf16x3_tensor", 1: "bf16x2_tensor", 2: "bf16_tensor"}
    fp32_hat = None
    for spec in args.variants.split(","):
        # "P": check-node precision P with the trellis channel node; "dP": the same with
        # the tensor-core (DFT) channel node
        dft = spec.startswith("d")
        prec = int(spec[1:] if dft else spec)
        ctx = jbp.Context(iters=50, early_stop=True, precision=prec,
                          channel_node=jbp.CHAN_DFT if dft else jbp.CHAN_TRELLIS)
        dec = jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"])
        dec.decode_device(y, hat, it, ok, form=jbp.FORM_STEP, stream=st)
        sec = _timed(torch, st, lambda: dec.decode_device(y, hat, it, ok, form=jbp.FORM_STEP, stream=st), 1)
        g = hat.cpu().numpy()
        if prec == 0 and not dft:
            fp32_hat = g
        m = torch.from_numpy(v2c).to(dev)
        dec.step_check(m, precision=prec, stream=st)
        st.synchronize()
        c2v_g = np.log(m.cpu().numpy().astype(np.float64))
        rho = np.exp(c2v_o)
        variants[("dft_channel+" if dft else "") + names[prec]] = {
            "frames_per_s": F / sec, "ms_per_batch": sec * 1e3, "mean_iters": float(it.float().mean().item()),
            "ser": float((g != fr["c"]).mean()),
            "ser_delta_vs_fp32": (float((g != fr["c"]).mean() - (fp32_hat != fr["c"]).mean())
                                  if fp32_hat is not None else None),
            "ser_oracle_sample": float((ref["hat"] != fr["c"][:S]).mean()) if ref else None,
            "ser_gpu_sample": float((g[:S] != fr["c"][:S]).mean()) if ref else None,
            "decisions_differing_from_oracle_at_margin_gt_1e-6": (int(((g[:S] != ref["hat"]) & (ref["margin"] > 1e-6)).sum())
                                                                 if ref else None),
            "check_step_max_log_err_rho_ge_0.5": float(np.abs(c2v_g - c2v_o)[rho >= 0.5].max()),
            "check_step_max_log_err_rho_ge_1e-4": float(np.abs(c2v_g - c2v_o)[rho >= 1e-4].max()),
            "check_step_max_linear_err": float(np.abs(np.exp(c2v_g) - rho).max()),
            "tc_timeouts": dec.tc_timeouts()}
        dec.close()
        ctx.close()
    chan = channel_legs(jbp, torch, dev, O, I, code, K, q, n, fr, st, args) if args.channel_legs else None
    return {"metric": METRIC, "value": max(v["frames_per_s"] for v in variants.values()), "unit": "frames/s",
            "config": {"workload": "K=4 users, GF(64) regular (2,4) LDPC, n=512, SNR 14 dB, 50 iterations with "
                                   "syndrome early stop, %d frames, step form (messages in HBM)" % F},
            "dtype": "f32 messages; check transform per variant", "variants": variants, "channel_node": chan,
            "cpu_baseline": ({"value": S / t_or, "unit": "frames/s", "cores": cores, "kind": "oracle",
                              "sample": "first %d frames, 50 iterations" % S} if S > 0 else None)}


def channel_legs(jbp, torch, dev, O, I, code, K, q, n, fr, st, args):
    """The channel node alone (one step over Fs frames, messages resident in HBM):
    FP32 trellis vs the tensor-core DFT form, time per channel use, bytes moved,
    the share of channel uses the DFT form hands to the trellis, and its error
    against the FP64 oracle on a 2-frame sample."""
    Fs = min(int(fr["y"].shape[0]), args.channel_frames)
    E = code["P"] * 4
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    x = torch.randn((Fs, K, E, q), generator=gen, device=dev) * 3.0
    msg0 = torch.exp(x - x.amax(-1, keepdim=True)).clamp_min_(1e-12)
    del x
    y = torch.from_numpy(fr["y"][:Fs]).to(dev)
    ch2v = torch.empty((Fs, K, n, q), dtype=torch.float32, device=dev)
    uses = Fs * n
    algo_bytes = uses * (5 * K * q * 4 + 4)    # c2v of both edges in, ch2v out, v2c of both edges out, y in
    out = {"frames": Fs, "channel_uses": uses, "algorithmic_bytes": algo_bytes}
    for name, node in (("trellis", jbp.CHAN_TRELLIS), ("dft", jbp.CHAN_DFT)):
        ctx = jbp.Context(iters=1, early_stop=False, channel_node=node)
        dec = jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"])
        msg = msg0.clone()
        for _ in range(2):
            dec.step_channel(y, msg, ch2v, stream=st)
        st.synchronize()
        f0 = dec.log_fallbacks()
        sec = _timed(torch, st, lambda: dec.step_channel(y, msg, ch2v, stream=st), 3)
        f1 = dec.log_fallbacks()
        out[name] = {"ms": sec * 1e3, "ns_per_channel_use": sec / uses * 1e9,
                     "gbs": algo_bytes / sec / 1e9, "rows_to_trellis_per_step": (f1 - f0) / 3,
                     "tc_timeouts": dec.tc_timeouts()}
        if node == jbp.CHAN_DFT:
            rng = np.random.default_rng(5)
            c2v_lin = np.exp(I.random_log_messages(rng, (2, K, E), q, spread=3.0)).astype(np.float32)
            m = torch.from_numpy(c2v_lin).to(dev)
            chs = torch.empty((2, K, n, q), dtype=torch.float32, device=dev)
            dec.step_channel(y[:2], m, chs, stream=st)
            st.synchronize()
            ch_o = np.exp(O.step_channel(code, K, fr["sigma2"], fr["perm"], fr["y"][:2],
                                         np.log(c2v_lin.astype(np.float64))))
            out[name]["max_linear_err_vs_oracle_2_frames"] = float(np.abs(chs.cpu().numpy() - ch_o).max())
        dec.close()
        ctx.close()
    out["speedup_dft_vs_trellis"] = out["trellis"]["ms"] / out["dft"]["ms"]
    return out


def _uneven_classes(F, seed):
    rng = np.random.default_rng(seed)
    Ks = rng.integers(2, 9, F)
    ns = rng.choice([128, 256, 512, 1024, 2048], F)
    qs = rng.choice([16, 64], F)
    snr = rng.uniform(8.0, 16.0, F)
    classes = {}
    for f in range(F):
        classes.setdefault((int(ns[f]), int(qs[f]), int(Ks[f])), []).append(f)
    return classes, snr


_FRAME_CACHE = {}


def _uneven_inputs(jbp, torch, dev, ctx, classes, snr):
    from paper_2605_26580_gb300 import inputs as I
    parts = []
    for (n, q, K), idx in sorted(classes.items()):
        Fc = len(idx)
        key = (n, q, K, Fc, tuple(idx[:4]))
        if key not in _FRAME_CACHE:
            code = _FRAME_CACHE.setdefault((n, q), None) or I.make_code(n, q)
            _FRAME_CACHE[(n, q)] = code
            fr = I.make_frames(code, K, 12.0, Fc, seed=4_000_000_000 + n * 1000 + q * 10 + K, device=dev)
            y, sig = I.channel_output(q, fr["c"], fr["perm"], snr[idx], 4_100_000_000 + n * 1000 + q * 10 + K)
            _FRAME_CACHE[key] = (code, fr, y, sig)
        code, fr, y, sig = _FRAME_CACHE[key]
        dec = jbp.Decoder(ctx, code, K, float(np.mean(sig)), fr["perm"])
        parts.append({"dec": dec, "c": fr["c"], "K": K, "n": n, "q": q, "F": Fc, "y": torch.from_numpy(y).to(dev),
                      "sig": torch.from_numpy(np.asarray(sig, np.float32)).to(dev),
                      "hat": torch.empty((Fc, K, n), dtype=torch.uint8, device=dev),
                      "it": torch.empty((Fc,), dtype=torch.int32, device=dev),
                      "ok": torch.empty((Fc, K), dtype=torch.uint8, device=dev),
                      "state": dec.state_bytes, "fused": dec.fused_ok})
    return parts


def _waves(parts, budget):
    """Group whole classes into waves whose HBM message state fits the budget."""
    waves, cur, used = [], [], 0
    for p in sorted(parts, key=lambda p: -p["state"] * p["F"] * (0 if p["fused"] else 1)):
        need = 0 if p["fused"] else p["state"] * p["F"]
        if cur and used + need > budget:
            waves.append(cur)
            cur, used = [], 0
        cur.append(p)
        used += need
    if cur:
        waves.append(cur)
    return waves


def _channel_node(jbp, args):
    return {"trellis": jbp.CHAN_TRELLIS, "dft": jbp.CHAN_DFT, "auto": jbp.CHAN_AUTO}[args.channel_node]


def wl_uneven(args):
    """100,000 frames with K ~ U{2..8}, n ~ U{128,...,2048}, q ~ U{16,64}, SNR ~ U[8,16] dB
    (per frame), 50 iterations with per-frame early stop.  Classes of equal
    (n, K, q) run concurrently; each memory wave is one jbp_decode_many call,
    captured as one CUDA graph and replayed; fused launch shapes autotuned."""
    jbp, torch, dev = _ctx_dev()
    F = int(100000 * args.frac)
    classes, snr = _uneven_classes(F, 404)
    ctx = jbp.Context(iters=50, early_stop=True, channel_node=_channel_node(jbp, args))
    t0 = time.perf_counter()
    parts = _uneven_inputs(jbp, torch, dev, ctx, classes, snr)
    t_gen = time.perf_counter() - t0
    budget = int(float(os.environ.get("JBP_BENCH_WAVE_GB", "60")) * 1e9)
    waves = _waves(parts, budget)
    st = torch.cuda.Stream()

    def one_pass():
        for w in waves:
            ctx.decode_many([(p["dec"], p["y"], p["hat"], p["it"], p["ok"], p["sig"]) for p in w], stream=st)

    t0 = time.perf_counter()
    one_pass()                     # eager + autotune
    one_pass()                     # capture
    st.synchronize()
    t_setup = time.perf_counter() - t0
    steps = max(1, min(args.steps, 3))
    sec = _timed(torch, st, one_pass, steps)   # graph replays
    ser_num = ser_den = 0
    iters = 0.0
    for p in parts:
        g = p["hat"].cpu().numpy()
        ser_num += int((g != p["c"]).sum())
        ser_den += g.size
        iters += float(p["it"].double().sum().item())
    fused_frames = sum(p["F"] for p in parts if p["fused"])
    out = {"metric": METRIC, "value": F / sec, "unit": "frames/s",
           "config": {"workload": "uneven batch: %d frames, K~U{2..8}, n~U{128,256,512,1024,2048}, q~U{16,64}, "
                                  "SNR~U[8,16] dB per frame, 50 iterations with per-frame early stop" % F,
                      "classes": len(parts), "waves": len(waves), "wave_budget_gb": budget / 1e9,
                      "channel_node": args.channel_node,
                      "graph": "one CUDA graph per wave (jbp_decode_many replay)"},
           "dtype": "f32", "s_per_batch": sec, "ser": ser_num / ser_den, "mean_iters": iters / F,
           "frames_fused_form": fused_frames, "frames_step_form": F - fused_frames,
           "setup_s": {"inputs": t_gen, "eager_tune_capture": t_setup}}
    for p in parts:
        p["dec"].close()
    ctx.close()
    return out


def steady_rate(done_t, t_first, n_req):
    """Saturated serving throughput.  done_t: completion times (s) of the requests
    that finished after the first poll sweep at t_first (the sweep that collects,
    at one time stamp, what finished while requests were still being submitted).
    Under overload the queue still holds most requests then: the completion rate
    from t_first until 90 % of all n_req requests are done is the engine's
    saturated throughput, without the drain at the end (pools emptying).  None
    when fewer than half the requests were still queued, or fewer than 100
    completions fall in that window.  Returns (frames/s, [t_first, t90])."""
    n90 = int(0.9 * n_req) - (n_req - len(done_t))
    if len(done_t) < n_req // 2 or n90 < 100:
        return None
    t90 = sorted(done_t)[n90 - 1]
    return n90 / max(1e-9, t90 - t_first), [t_first, t90]


def wl_serve(args):
    """Serving: Poisson arrivals of single frames drawn from the uneven-batch size
    distribution, continuous batching over concurrent launches with admission by
    memory budget; frames/s and p50/p99 submit-to-result latency per arrival rate,
    and the plain per-frame form's latency for comparison."""
    jbp, torch, dev = _ctx_dev()
    N = int(20000 * args.frac)
    classes, snr = _uneven_classes(N, 505)
    # the workload's rates (20K-200K requests/s, above this mix's capacity) and
    # rates below it, where latency is service time rather than queueing; a rate
    # below the knee runs about 4 s of arrivals
    rates = [int(r) for r in str(args.rates).split(",") if r]
    results = []
    for lam in rates:
        ctx = jbp.Context(iters=50, early_stop=True, mem_budget_bytes=int(64e9),
                          channel_node=_channel_node(jbp, args), block_iters=args.block_iters)
        parts = _uneven_inputs(jbp, torch, dev, ctx, classes, snr)
        reqs = []
        for p in parts:
            yh = p["y"].cpu().numpy()
            sh = p["sig"].cpu().numpy()
            for i in range(p["F"]):
                reqs.append((p, i, yh[i], float(sh[i])))
        n_req = min(len(reqs), max(200, int(4 * lam)))
        order = np.random.default_rng(lam).permutation(len(reqs))[:n_req]
        gaps = np.random.default_rng(lam + 1).exponential(1.0 / lam, n_req)
        tickets = []
        t_start = time.perf_counter()
        t_next = t_start
        for j, r in enumerate(order):
            t_next += gaps[j]
            while time.perf_counter() < t_next:
                pass
            p, i, yv, sv = reqs[r]
            tickets.append((p, i, p["dec"].submit(yv, sv)))
        t_sub = time.perf_counter() - t_start
        ser_num = ser_den = 0
        pending = list(tickets)
        # completion times after the first sweep (that sweep collects what finished
        # while requests were still being submitted, at one time stamp)
        done_t, t_first = [], None
        while pending:
            rest = []
            for p, i, tk in pending:
                res = ctx.poll(tk, p["n"], p["K"])
                if res is None:
                    rest.append((p, i, tk))
                else:
                    if t_first is not None:
                        done_t.append(time.perf_counter() - t_start)
                    ser_num += int((res["hat"] != p["c"][i]).sum())
                    ser_den += res["hat"].size
            if t_first is None:
                t_first = time.perf_counter() - t_start
            pending = rest
        wall = time.perf_counter() - t_start
        stats = ctx.serving_stats()
        row = {"offered_req_per_s": lam, "requests": n_req, "achieved_submit_rate": n_req / t_sub,
               "frames_per_s": n_req / wall, "p50_ms": stats["p50_us"] / 1e3,
               "p99_ms": stats["p99_us"] / 1e3, "ser": ser_num / max(1, ser_den),
               "completed": stats["completed"]}
        st = steady_rate(done_t, t_first, n_req)
        if st is not None:
            row["steady_frames_per_s"], row["steady_window_s"] = st
        results.append(row)
        for p in parts:
            p["dec"].close()
        ctx.close()
    # plain per-frame form: one frame per launch sequence, no batching
    ctx = jbp.Context(iters=50, early_stop=True)
    parts = _uneven_inputs(jbp, torch, dev, ctx, dict(list(classes.items())[:6]), snr)
    lat = []
    for p in parts:
        yh = p["y"].cpu().numpy()
        for i in range(min(3, p["F"])):
            t0 = time.perf_counter()
            p["dec"].decode(yh[i:i + 1], form=jbp.FORM_PLAIN)
            lat.append(time.perf_counter() - t0)
    for p in parts:
        p["dec"].close()
    ctx.close()
    best = max(results, key=lambda r: r["frames_per_s"])
    steady = [r["steady_frames_per_s"] for r in results if "steady_frames_per_s" in r]
    return {"metric": METRIC, "value": best["frames_per_s"], "unit": "frames/s",
            "config": {"workload": "serving: %d single-frame requests per rate, sizes from the uneven-batch "
                                   "distribution, Poisson arrivals" % N, "rates": rates,
                       "block_iters": args.block_iters or 5},
            "dtype": "f32", "per_rate": results,
            "saturation_steady_frames_per_s": max(steady) if steady else None,
            "plain_per_frame_form": {"p50_ms": 1e3 * float(np.median(lat)), "frames_per_s": len(lat) / sum(lat),
                                     "sample": "%d frames from 6 classes, one launch sequence each" % len(lat)}}


# FFT-BP ms/sample of the paper's Table 1 (K=2, Q=64, R=1/3; SIC with WHT check nodes on
# AMP evidence, 50 iterations with early exit; RTX 3090 / i5-14500, precision not stated)
PAPER_FFT_BP_MS = {12: 8.34, 18: 15.19, 24: 59.59, 48: 767.51}
# the same for the PEG-LDPC code at Q=64, L=12 (the paper's PEG-LDPC comparison table)
PAPER_PEG_FFT_BP_MS = 7.99


def sic_flops_per_row_iter(n, P, dc, q):
    """Algorithmic FLOPs of one BP iteration of one row: per check dc forward and
    dc inverse WHTs (q log2 q add/sub each) and about 4 dc q multiplies
    (leave-one-out products, floor, scale); per variable 6 q multiplies."""
    return P * dc * q * (2 * int(math.log2(q)) + 4) + 6 * n * q


def amp_flops_per_slot_iter(q):
    """Two radix-2 transforms of length q (q/2 log2 q butterflies of 10 FLOPs) and
    about 30 FLOPs of denoiser per coordinate."""
    return 2 * (q // 2) * int(math.log2(q)) * 10 + 30 * q


def wl_ura(args):
    """The paper's own classical path on the evidence interface (Table 1 shapes):
    K=2 rows, GF(64) regular (2,3) codes of rate 1/3, L in {12, 18, 24, 48} slots,
    ns = 24 partial-DFT rows per slot, E_b/N_0 = 10 dB, AMP 20 iterations, SIC over
    2 rows of FFT-BP with at most 50 iterations and early exit.  Times the slot
    detector, the SIC decoder (the part the paper's FFT-BP time covers) and both,
    the single-frame latency, matched SER/CER, and the oracle on a sample."""
    jbp, torch, dev = _ctx_dev()
    from oracle import oracle as O
    from paper_2605_26580_gb300 import inputs as I
    K, q, ns, eb = 2, 64, 24, 10.0
    cores = os.cpu_count() or 1
    st = torch.cuda.Stream()
    per_L = []
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp32_peak_tflops(sm, 2070.0)
    for L, family in ((12, "random"), (18, "random"), (24, "random"), (48, "random"), (12, "peg")):
        F = int((131072 if L < 48 else 65536) * args.frac)
        code = I.make_code(L, q, dv=2, dc=3) if family == "random" else I.make_peg_code(L, q)
        chunks = [I.make_ura_frames(code, K, eb, min(16384, F - c), seed=4_000_000_000 + L * 1000 + c // 16384)
                  for c in range(0, F, 16384)]
        fr0 = chunks[0]
        X = np.concatenate([c["X"] for c in chunks])
        y = torch.from_numpy(np.concatenate([c["y"] for c in chunks])).to(dev)
        ctx = jbp.Context(iters=50)
        dec = jbp.EvidenceDecoder(ctx, code, K, fr0["rows"], fr0["rho"], fr0["su2"], fr0["cancel_log"])
        S = torch.empty((F, L, q), dtype=torch.float32, device=dev)
        hat = torch.empty((F, K, L), dtype=torch.uint8, device=dev)
        it = torch.empty((F, K), dtype=torch.int32, device=dev)
        ok = torch.empty((F, K), dtype=torch.uint8, device=dev)
        for _ in range(3):
            dec.decode_device(y, hat, it, ok, stream=st)
            dec.evidence_device(y, S, stream=st)
            dec.sic_device(S, hat, it, ok, stream=st)
        steps = max(3, args.steps)
        t_amp = _timed(torch, st, lambda: dec.evidence_device(y, S, stream=st), steps)
        t_sic = _timed(torch, st, lambda: dec.sic_device(S, hat, it, ok, stream=st), steps)
        t_all = _timed(torch, st, lambda: dec.decode_device(y, hat, it, ok, stream=st), steps)
        t_one = _timed(torch, st, lambda: dec.sic_device(S[:1], hat[:1], it[:1], ok[:1], stream=st), 20)
        t_one_all = _timed(torch, st, lambda: dec.decode_device(y[:1], hat[:1], it[:1], ok[:1], stream=st), 20)
        # end to end through the host API: y from pinned host memory, rows back to the host
        yh = y.cpu().pin_memory()
        t0 = time.perf_counter()
        host = dec.decode(yh.numpy())
        t_e2e = time.perf_counter() - t0
        g = hat.cpu().numpy()
        iters = it.cpu().numpy()
        # row-aligned errors on the GPU (jbp_match_rows), checked against the host on a sample
        Xd = torch.from_numpy(X).to(dev)
        sym_d = torch.empty((F,), dtype=torch.int32, device=dev)
        cw_d = torch.empty((F,), dtype=torch.int32, device=dev)
        ctx.match_rows_device(hat, Xd, sym_d, cw_d, stream=st)
        st.synchronize()
        sym, cw = sym_d.cpu().numpy(), cw_d.cpu().numpy()
        hs, hc = I.match_rows(g[:4096], X[:4096])
        match_ok = bool(np.array_equal(hs, sym[:4096]) and np.array_equal(hc, cw[:4096]))
        P = code["P"]
        fl_sic = float(iters.sum()) * sic_flops_per_row_iter(L, P, 3, q)
        fl_amp = float(F) * L * 21 * amp_flops_per_slot_iter(q)
        # oracle on a bounded sample (all host cores)
        So = min(F, max(64, int(2048 * 12 / L)))
        t0 = time.perf_counter()
        Sref = O.amp_evidence(q, fr0["rows"], y[:So].cpu().numpy(), 20, fr0["rho"], fr0["su2"], threads=cores)
        t_or_amp = time.perf_counter() - t0
        t0 = time.perf_counter()
        ref = O.sic_decode(code, K, S[:So].cpu().numpy().astype(np.float64), 50, fr0["cancel_log"], threads=cores)
        t_or_sic = time.perf_counter() - t0
        same = (ref["hat"] == g[:So]) | (ref["margin"] <= 1e-6)
        dec.close()
        ctx.close()
        per_L.append({
            "L": L, "P": P, "code": family, "girth": I.girth(code), "frames": F, "sic_frames_per_s": F / t_sic, "amp_frames_per_s": F / t_amp,
            "pipeline_frames_per_s": F / t_all, "e2e_frames_per_s": F / t_e2e,
            "sic_ms_per_sample_amortised": 1e3 * t_sic / F, "sic_latency_ms_single_frame": 1e3 * t_one,
            "pipeline_latency_ms_single_frame": 1e3 * t_one_all,
            "paper_fft_bp_ms_per_sample": PAPER_FFT_BP_MS[L] if family == "random" else PAPER_PEG_FFT_BP_MS,
            "ser": float(sym.sum() / X.size), "cer": float(cw.sum() / (F * K)), "gpu_matching_equals_host": match_ok,
            "mean_bp_iters_per_row": [float(v) for v in iters.mean(0)], "rows_ok": float(ok.float().mean().item()),
            "sic_roofline": {"bound": "alu", "achieved": fl_sic / t_sic / 1e12, "peak": peak, "unit": "TFLOP/s",
                             "frac": fl_sic / t_sic / 1e12 / peak},
            "amp_roofline": {"bound": "alu", "achieved": fl_amp / t_amp / 1e12, "peak": peak, "unit": "TFLOP/s",
                             "frac": fl_amp / t_amp / 1e12 / peak},
            "oracle": {"frames": So, "cores": cores, "amp_frames_per_s": So / t_or_amp,
                       "sic_frames_per_s": So / t_or_sic,
                       "decisions_differing_at_margin_gt_1e-6": int((~same).sum())},
        })
    best = per_L[0]
    return {"metric": METRIC, "value": best["sic_frames_per_s"], "unit": "frames/s",
            "config": {"workload": "evidence interface (Table 1 shapes): K=2, GF(64) regular (2,3) LDPC of rate 1/3, "
                                   "L in {12,18,24,48}, ns=24 partial-DFT rows per slot, Eb/N0 10 dB, AMP 20 "
                                   "iterations, SIC over 2 rows of FFT-BP (<= 50 iterations, early exit); also the PEG "
                                   "code at L=12; value = SIC decoder frames/s at L=12",
                       "l2": "inputs (y and S) of every L are larger than the 129 MB L2"},
            "dtype": "f32", "data": "synthetic", "per_L": per_L}


if __name__ == "__main__":
    main()
