#!/usr/bin/env python
"""Throughput benchmark of batched NDGSBP decoding on GB300.

Workload (one "step"): the n=2304 rate-1/2 QC-LDPC code (12x24 base matrix, Z=96, VN degrees
{2,3,6}), NDGSBP over 12 cyclic windows of 2 layers (overlap 1 layer), FP32 edge messages,
I_max 25 (the check-update budget of 50 flooding iterations), a sweep of 9 Eb/N0 points
0.5..2.5 dB with 65,536 frames per point per GPU.  Per point the step generates the channel
LLRs on the GPU (Philox/Box-Muller, all-zero codeword) and decodes them with the fused
statistics epilogue.  Decoded throughput counts K = N - M = 1152 information bits per frame.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a bounded sample
of the same workload on the host cores.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NDGSBP decoded Gbit/s and p50/p99 frame latency at oracle-matched FER"
CODE_NAME = "qc_n2304_r12"
EBN0 = [0.5 + 0.25 * i for i in range(9)]
FRAMES = 65536
IMAX_ND = 25
IMAX_FLOOD = 50
GROUP_SEED = 2304
CHANNEL_SEED = 0x5EED0000
RATE = 0.5
MUFU_PER_EDGE_UPDATE = 3          # exp2, reciprocal, log2 per edge of Eq. (1)
MUFU_PER_CLK_PER_SM = 32          # MUFU results per clock per SM sustained on GB300 (one warp
                                  # instruction per clock per SM, the XU-pipe peak ncu normalises to)
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "decode_qc_n2304_traffic.json")


def workload_config(frames):
    return {
        "workload": "qc_n2304_r12 NDGSBP 12 cyclic 2-layer groups (overlap 1 layer), FP32 messages, "
                    "I_max 25, Eb/N0 0.5..2.5 dB step 0.25, channel LLRs generated on the GPU",
        "code": CODE_NAME, "N": 2304, "K": 1152, "Z": 96, "frames_per_point": frames,
        "ebn0_db": EBN0, "points": len(EBN0), "max_iter": IMAX_ND, "msg_dtype": "f32",
        "schedule": "NDGSBP", "groups": 12, "overlap_layers": 1,
        "l2": "inputs larger than L2: 604 MB of LLRs per point",
        "parallelism": "frame-sharded replicas",
    }


# ------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sms, maxes, powers, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sms.append(float(parts[1]))
                    maxes.append(float(parts[2]))
                    powers.append(float(parts[3]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        top = max(sms)
        loaded = [s for s in sms if s >= 0.5 * top] or sms
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(maxes), "samples": len(sms),
                "power_w_max": max(powers), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for fn in ("decode.cu", "decode_qc.cu"):
        p = os.path.join(ROOT, "paper_1202_1060_gb300", "csrc", fn)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    try:
        with open(PROFILE_TRAFFIC) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None, None
    if rec.get("source_hash") != kernel_source_hash() or rec.get("kernel") != kernel_name:
        return None, rec
    return rec.get("dram_bytes_per_launch_full"), rec


# ------------------------------------------------------------------------------------------
# CPU oracle leg
# ------------------------------------------------------------------------------------------
def oracle_sweep(frames_per_point, threads=None, seed_base=CHANNEL_SEED):
    """Decode frames_per_point frames at every Eb/N0 point with the FP64 oracle (its own channel
    generator, same definition and seeds as the GPU generator).  Returns (seconds, frames, errors
    per point)."""
    from oracle import oracle as O
    from paper_1202_1060_gb300 import inputs as I
    code = I.code_by_name(CODE_NAME)
    gp, gc = O.groups(code.M, 12, 0.5, GROUP_SEED, unit=code.Z, cyclic=True)
    llrs = [O.awgn_llr(code.N, frames_per_point, eb, RATE, seed_base + i) for i, eb in enumerate(EBN0)]
    fe = []
    t0 = time.perf_counter()
    for llr in llrs:
        r = O.ndgsbp_decode(code, gp, gc, llr, IMAX_ND, want_total=False, n_threads=threads)
        fe.append(int(r.hard.any(axis=1).sum()))
    dt = time.perf_counter() - t0
    return dt, frames_per_point * len(EBN0), fe


def clopper_pearson(k, n, alpha=0.05):
    from scipy import stats
    lo = 0.0 if k == 0 else float(stats.beta.ppf(alpha / 2, k, n - k + 1))
    hi = 1.0 if k == n else float(stats.beta.ppf(1 - alpha / 2, k + 1, n - k))
    return lo, hi


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    """--impl reference: the FP64 oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    per_point = args.ref_frames
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sweep(max(1, per_point // 4))
    times = []
    for s in range(args.steps):
        dt, nf, _ = oracle_sweep(per_point, seed_base=CHANNEL_SEED + 1000 * s)
        times.append(dt)
    total = sum(times)
    frames = per_point * len(EBN0) * args.steps
    value = frames * 1152 / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(per_point),
        "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_point} frames per Eb/N0 point x {len(EBN0)} points per step"},
        "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# GPU leg
# ------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import inputs as I
    from paper_1202_1060_gb300 import ndgsbp as nd

    c = I.code_by_name(CODE_NAME)
    code = nd.Code.from_inputs(c)
    groups = nd.Groups.build(code, 12, 0.5, GROUP_SEED, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
    params = nd.params_default(max_iter=IMAX_ND, msg_dtype=nd.F32, variant=args.variant)
    F = args.frames
    W = (c.N + 31) // 32
    plan = groups.plan(params, F)
    q = groups.query()
    edge_updates_iter = q["edge_updates_per_iter"]
    stream = torch.cuda.Stream(device=dev)
    llr = torch.empty((F, c.N), dtype=torch.float32, device=dev)
    ws = torch.zeros(max(256, groups.workspace_size(params, F)), dtype=torch.uint8, device=dev)
    hard = torch.empty((F, W), dtype=torch.int32, device=dev)
    iters = torch.empty(F, dtype=torch.int32, device=dev)
    ok = torch.empty(F, dtype=torch.uint8, device=dev)
    stats = torch.zeros((len(EBN0), nd.STATS_LEN), dtype=torch.int64, device=dev)
    hist = torch.zeros(IMAX_ND + 1, dtype=torch.int64, device=dev)
    start_ns = torch.zeros(F, dtype=torch.int64, device=dev)
    retire_ns = torch.zeros(F, dtype=torch.int64, device=dev)

    def step(s, timing=None, latency=False):
        for i, eb in enumerate(EBN0):
            seed = CHANNEL_SEED + i + 1000 * s + (rank << 40)
            nd.awgn_llr(code, F, eb, RATE, seed, llr, stream=stream)
            if timing is not None:
                timing.append(torch.cuda.Event(enable_timing=True))
                timing[-1].record(stream)
            nd.decode(groups, params, llr, ws, hard, iters, ok, stats=stats[i], iter_hist=hist,
                      start_ns=start_ns if latency else None, retire_ns=retire_ns if latency else None,
                      stream=stream)
            if timing is not None:
                timing.append(torch.cuda.Event(enable_timing=True))
                timing[-1].record(stream)

    # warm-up
    for s in range(args.warmup):
        step(-1 - s)
    torch.cuda.synchronize()
    stats.zero_()
    hist.zero_()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    dec_events = []
    ev0.record(stream)
    for s in range(args.steps):
        step(s, timing=dec_events, latency=(s == args.steps - 1))
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    clk = clocks.stop()
    dec_ms = [dec_events[2 * j].elapsed_time(dec_events[2 * j + 1]) for j in range(len(dec_events) // 2)]
    t = torch.tensor([elapsed], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    elapsed_max = float(t.item())
    frames_total = F * len(EBN0) * args.steps * world
    value = frames_total * 1152 / elapsed_max / 1e9

    st = stats.cpu().numpy()
    frames_done = int(st[:, nd.STAT_FRAMES].sum())
    iter_sum = int(st[:, nd.STAT_ITERATIONS].sum())
    fer = (st[:, nd.STAT_FRAME_ERRORS] / np.maximum(st[:, nd.STAT_FRAMES], 1)).tolist()
    ber = (st[:, nd.STAT_BIT_ERRORS] / np.maximum(st[:, nd.STAT_FRAMES] * c.N, 1)).tolist()

    # latency of the last timed point (frames of one decode launch)
    s_ns = start_ns.cpu().numpy().astype(np.float64)
    r_ns = retire_ns.cpu().numpy().astype(np.float64)
    service = (r_ns - s_ns) / 1e6
    batch = (r_ns - s_ns.min()) / 1e6

    # roofline of the decode kernel: MUFU operations (3 per edge-update) over its launch time
    peaks, peak_kind = measured_peaks()
    dec_total_s = sum(dec_ms) / 1e3
    mufu_ops = MUFU_PER_EDGE_UPDATE * edge_updates_iter * iter_sum
    achieved = mufu_ops / dec_total_s / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = MUFU_PER_CLK_PER_SM * sms * peak_clock_mhz * 1e6 / 1e12
    kname = {nd.VARIANT_QC: "qc_decode_kernel", nd.VARIANT_QC_GLOBAL: "qc_decode_kernel",
             nd.VARIANT_QC_PAIR: "qc_pair_kernel", nd.VARIANT_QC_PAIR_GLOBAL: "qc_pair_kernel"}.get(plan.variant,
                                                                                            "decode_kernel")
    traffic, traffic_rec = profiled_traffic(kname)
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s", "frac": achieved / peak,
        "traffic": traffic,
        "what": f"MUFU ops (exp2+rcp+lg2 = {MUFU_PER_EDGE_UPDATE} per edge-update of Eq. (1)) of the decode "
                f"kernel over its CUDA-event time; peak = {MUFU_PER_CLK_PER_SM} MUFU/clk/SM x {sms} SMs x "
                f"{peak_clock_mhz:.0f} MHz (clock from MEASURED_PEAKS.json, {peak_kind})",
        "kernel": kname, "launches": len(dec_ms), "avg_launch_ms": sum(dec_ms) / len(dec_ms),
        "edge_updates_per_launch": edge_updates_iter * iter_sum / len(dec_ms),
        "hbm_bytes_per_launch_algorithmic": F * (c.N * 4 + W * 4 + 5),
        "hbm_frac_of_measured": F * (c.N * 4 + W * 4 + 5) / (sum(dec_ms) / len(dec_ms) / 1e3) / 1e9 / peaks["hbm_gbs"],
    }

    # end-to-end through host buffers: pinned host LLRs -> device -> decode -> decisions back
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, nd, torch, code, c, groups, params, F, W, dev, rank, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        dt, nf, fe_or = oracle_sweep(args.cpu_frames)
        cpu = {"value": nf * 1152 / dt / 1e9, "unit": "Gbit/s", "cores": host_cores(), "kind": "oracle",
               "sample": f"{args.cpu_frames} frames at each of the {len(EBN0)} Eb/N0 points (same channel "
                         f"definition and seeds), {dt:.1f} s", "seconds": dt}
        # FER agreement on the frames both decoded (the first cpu_frames of each point of step 0
        # are generated from the same seeds): GPU FER must sit inside the oracle's 95% interval
        fer_ci = []
        for i in range(len(EBN0)):
            lo, hi = clopper_pearson(fe_or[i], args.cpu_frames)
            fer_ci.append([lo, hi])
        cpu["oracle_fer"] = [f / args.cpu_frames for f in fe_or]
        cpu["oracle_fer_ci95"] = fer_ci
        cpu["gpu_fer_inside_ci"] = all(lo <= g <= hi for g, (lo, hi) in zip(fer, fer_ci))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(F),
            "latency": {"p50_ms": float(np.percentile(service, 50)), "p99_ms": float(np.percentile(service, 99)),
                        "batch_p50_ms": float(np.percentile(batch, 50)),
                        "batch_p99_ms": float(np.percentile(batch, 99)),
                        "what": "service = frame retire - frame start; batch = frame retire - launch start "
                                "(last timed decode launch, 65,536 frames at 2.5 dB)"},
            "fer": fer, "ber": ber, "mean_iterations": iter_sum / max(frames_done, 1),
            "mean_iterations_per_point": (st[:, nd.STAT_ITERATIONS] / np.maximum(st[:, nd.STAT_FRAMES], 1)).tolist(),
            "coded_gbit_s": frames_total * c.N / elapsed_max / 1e9,
            "clocks": clk, "gpu_launches": 2 * len(EBN0) * args.steps,
            "plan": plan.as_dict(), "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_e2e(args, nd, torch, code, c, groups, params, F, W, dev, rank, world):
    """Same metric through the public API with host buffers: every step copies each point's
    LLRs from pinned host memory, decodes, and copies decisions, iteration counts and syndrome
    flags back.  Copies of the next point overlap the current decode (two streams)."""
    import numpy as np
    import torch.distributed as dist
    n_pts = len(EBN0)
    host_llr = []
    tmp = torch.empty((F, c.N), dtype=torch.float32, device=dev)
    for i, eb in enumerate(EBN0):
        nd.awgn_llr(code, F, eb, RATE, CHANNEL_SEED + 77 + i + (rank << 40), tmp)
        h = torch.empty((F, c.N), dtype=torch.float32, pin_memory=True)
        h.copy_(tmp)
        host_llr.append(h)
    del tmp
    host_hard = torch.empty((n_pts, F, W), dtype=torch.int32, pin_memory=True)
    host_iters = torch.empty((n_pts, F), dtype=torch.int32, pin_memory=True)
    host_ok = torch.empty((n_pts, F), dtype=torch.uint8, pin_memory=True)
    d_llr = [torch.empty((F, c.N), dtype=torch.float32, device=dev) for _ in range(2)]
    d_hard = [torch.empty((F, W), dtype=torch.int32, device=dev) for _ in range(2)]
    d_iters = [torch.empty(F, dtype=torch.int32, device=dev) for _ in range(2)]
    d_ok = [torch.empty(F, dtype=torch.uint8, device=dev) for _ in range(2)]
    ws = torch.zeros(max(256, groups.workspace_size(params, F)), dtype=torch.uint8, device=dev)
    copy_s = torch.cuda.Stream(device=dev)
    comp_s = torch.cuda.Stream(device=dev)

    def one_step():
        loaded = [torch.cuda.Event() for _ in range(n_pts)]
        done = [torch.cuda.Event() for _ in range(n_pts)]
        for i in range(n_pts):
            b = i % 2
            with torch.cuda.stream(copy_s):
                if i >= 2:
                    copy_s.wait_event(done[i - 2])
                d_llr[b].copy_(host_llr[i], non_blocking=True)
                loaded[i].record(copy_s)
            with torch.cuda.stream(comp_s):
                comp_s.wait_event(loaded[i])
                nd.decode_plain(groups, params, d_llr[b], ws, d_hard[b], d_iters[b], d_ok[b], stream=comp_s)
                host_hard[i].copy_(d_hard[b], non_blocking=True)
                host_iters[i].copy_(d_iters[b], non_blocking=True)
                host_ok[i].copy_(d_ok[b], non_blocking=True)
                done[i].record(comp_s)

    for _ in range(max(1, args.warmup)):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    dt = time.perf_counter() - t0
    t = torch.tensor([dt], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dt = float(t.item())
    frames = F * n_pts * args.steps * world
    h2d = n_pts * F * c.N * 4
    d2h = n_pts * F * (W * 4 + 4 + 1)
    ok_frac = float(host_ok.float().mean())
    return {"value": frames * 1152 / dt / 1e9, "unit": "Gbit/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * dt / args.steps,
            "timer": "host wall clock around all steps, synchronised", "syndrome_ok_fraction": ok_frac}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=FRAMES, help="frames per Eb/N0 point per GPU")
    ap.add_argument("--variant", type=int, default=0, help="decode variant (0 = library choice)")
    ap.add_argument("--cpu-frames", type=int, default=512, help="oracle sample per Eb/N0 point")
    ap.add_argument("--ref-frames", type=int, default=64, help="oracle frames per point per reference step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
