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


def hbm_peak_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


# --------------------------------------------------------------------------- reference arm (the oracle)

def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    from paper_2605_26580_gb300 import inputs as I
    cores = os.cpu_count() or 1
    S = args.ref_frames or max(4, cores)
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
    S = max(8, cores)
    code = I.make_code(N_SYM, Q)
    fr = I.make_frames(code, K_USERS, 10.0, S, seed=frame_seed(2, 0))
    t0 = time.perf_counter()
    O.decode(code, K_USERS, fr["sigma2"], fr["perm"], fr["y"], ITERS, early_stop=True, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": S / dt, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": "%d frames at 10 dB of the same workload, FP64 oracle, %d threads, %.1f s" % (S, cores, dt)}


# --------------------------------------------------------------------------- our arm

def main() -> None:
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
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
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
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * F * args.steps / (total_ms / 1e3)

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
    peak = fp32_peak_tflops(sm_count, 2070.0)
    achieved = flops / (total_ms / 1e3) / 1e12 / world
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "k_fused<16,4>",
                "peak_note": "FP32 FMA peak derived: %d SMs x 128 lanes x 2 flops x 2070 MHz" % sm_count,
                "flops_per_frame_iter": flops_per_frame_iter(K_USERS, Q, N_SYM)}

    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "K": K_USERS, "q": Q, "n": N_SYM, "frames_per_batch": F,
                   "iters": ITERS, "early_stop": True, "snr_db": SNRS, "form": args.form,
                   "l2": "inputs cycle through 6 batches x %.0f MB (> 129 MB L2); message state in shared memory"
                         % (F * N_SYM * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
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
    if rank == 0:
        print(json.dumps(line), flush=True)
    for d in decs:
        d.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()


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
    out["step_form"] = {"value": F / (ms / 1e3), "unit": "frames/s",
                        "matches_fused": bool(np.array_equal(hat.cpu().numpy(), res["hat"]))}
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


if __name__ == "__main__":
    main()
