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
# scratch files of a bench run (clock samples, the autotuner's cache); not part of the results
OUT_DIR = os.environ.get("NDGSBP_BENCH_OUT", os.path.join(ROOT, "bench_out"))
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
MUFU_PER_CLK_PER_SM = 32          # nominal MUFU results per clock per SM (one warp instruction per
                                  # clock per SM, the XU-pipe peak ncu normalises to); the roofline
                                  # uses the rate measured by ndgsbp_mufu_probe
LATENCY_POINT = 5                 # EBN0[5] = 1.75 dB, the FER ~ 1e-3 point of the n=2304 code
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "qc_decode_kernel_n2304_sweep.md")


def channel_seed(point, step, rank, base=CHANNEL_SEED):
    """Seed of one Eb/N0 point's channel LLRs in one step on one rank: frame-sharded replicas
    draw disjoint Philox streams (the rank sits in the seed's upper bits)."""
    return base + point + 1000 * step + (rank << 40)


def max_over_ranks(x, device, world):
    """The slowest rank's time: the whole job is done when the last rank is."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(t, world):
    """Error and iteration counters summed over the ranks' shards (in place)."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def whole_job_gbits(frames_per_rank, world, bits_per_frame, seconds):
    """Whole-job throughput: the frames of all ranks over the slowest rank's time."""
    return frames_per_rank * world * bits_per_frame / seconds / 1e9


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
        os.makedirs(OUT_DIR, exist_ok=True)
        self.path = os.path.join(OUT_DIR, f"clocks_{os.getpid()}.csv")

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


KERNEL_SOURCES = ("qc_kernel.cuh", "decode_qc.cu", "decode_qc.h", "qc_device.cuh", "device_common.cuh")


def kernel_source_hash():
    """Hash of the sources of the n=2304 decode kernel (qc_decode_kernel)."""
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES:
        p = os.path.join(ROOT, "paper_1202_1060_gb300", "csrc", fn)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_name):
    """DRAM bytes per full-size launch from the committed ncu summary (lines "key: value"), if it
    was taken on the current kernel source; else None."""
    rec = {}
    try:
        with open(PROFILE_TRAFFIC) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    rec[k.strip()] = v.strip().strip("`")
    except OSError:
        return None, None
    if rec.get("source_hash") != kernel_source_hash() or rec.get("kernel") != kernel_name:
        return None, rec
    try:
        return float(rec["dram_bytes_per_launch_full"]), rec
    except (KeyError, ValueError):
        return None, rec


# ------------------------------------------------------------------------------------------
# CPU oracle leg
# ------------------------------------------------------------------------------------------
def oracle_sweep(frames_per_point, threads=None, seed_base=CHANNEL_SEED, keep=None):
    """Decode frames_per_point frames at every Eb/N0 point with the FP64 oracle (its own channel
    generator, same definition and seeds as the GPU generator).  Returns (seconds, frames, errors
    per point); with keep a list, appends each point's oracle Result to it."""
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
        if keep is not None:
            keep.append(r)
    dt = time.perf_counter() - t0
    return dt, frames_per_point * len(EBN0), fe


def paired_check(nd, torch, code, c, groups, params, oracle_results, n, dev, stream):
    """The GPU decodes the same n frames per Eb/N0 point as the oracle (step 0's first n frames,
    same seeds) outside the timed region; counts, per point, the frames whose frame-error status,
    hard decisions or iteration counts differ from the oracle's (FP32 against FP64: differences
    are expected only on frames the oracle does not decode, whose trajectories are chaotic)."""
    import numpy as np
    W = (c.N + 31) // 32
    llr = torch.empty((n, c.N), dtype=torch.float32, device=dev)
    hard = torch.empty((n, W), dtype=torch.int32, device=dev)
    iters = torch.empty(n, dtype=torch.int32, device=dev)
    ws = torch.zeros(max(256, groups.workspace_size(params, n)), dtype=torch.uint8, device=dev)
    out = {"frames_per_point": n, "frame_error_status_differs": [], "bits_differ_frames": [],
           "iterations_differ": [], "oracle_failing": []}
    for i, (eb, ref) in enumerate(zip(EBN0, oracle_results)):
        nd.awgn_llr(code, n, eb, RATE, channel_seed(i, 0, 0), llr, stream=stream)
        nd.decode(groups, params, llr, ws, hard, iters, stream=stream)
        torch.cuda.synchronize()
        bits = nd.unpack_bits(hard, c.N)
        it = iters.cpu().numpy()
        out["frame_error_status_differs"].append(int((bits.any(axis=1) != ref.hard.any(axis=1)).sum()))
        out["bits_differ_frames"].append(int((bits != ref.hard).any(axis=1).sum()))
        out["iterations_differ"].append(int((it != ref.iters).sum()))
        out["oracle_failing"].append(int((ref.synd_ok == 0).sum()))
    return out


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
        "data": "synthetic", "config": workload_config(args.frames),
        "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
                         "sample": f"a bounded sample of the workload: {per_point} frames per Eb/N0 point x "
                                   f"{len(EBN0)} points per step (the workload has {args.frames} per point)"},
        "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# extras of the default line (outside its timed region)
# ------------------------------------------------------------------------------------------
def mufu_peak(nd, torch, dev, sms, sm_mhz, iters=8192):
    """Rates of ex2 / rcp / lg2 (.approx, FP32) from ndgsbp_mufu_probe on a full grid (2 CTAs of
    1024 threads per SM, 8 independent chains per thread), CUDA-event timed on the probe's stream,
    and the rate of the decode kernels' 1:1:1 mix (equal counts: the harmonic mean)."""
    blocks, threads = 2 * sms, 1024
    sink = torch.zeros(blocks, dtype=torch.float32, device=dev)
    st = torch.cuda.Stream(device=dev)
    out, inv = {}, 0.0
    for op, name in enumerate(("ex2", "rcp", "lg2")):
        nd.mufu_probe(op, iters // 8, blocks, threads, sink, stream=st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        nd.mufu_probe(op, iters, blocks, threads, sink, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        rate = blocks * threads * iters * 8 / sec
        inv += 1.0 / rate
        out[name] = {"tops": rate / 1e12, "per_clk_per_sm": rate / (sms * sm_mhz * 1e6), "ms": 1e3 * sec}
    mix = 3.0 / inv
    out.update({"mix_tops": mix / 1e12, "mix_per_clk_per_sm": mix / (sms * sm_mhz * 1e6), "sm_mhz": sm_mhz,
                "what": f"{blocks} x {threads} threads x {iters} rounds x 8 chains per op"})
    return out


def flood_equal_budget(nd, torch, dev, code, c, F, stream, rank):
    """Flooding at I_max 50 beside NDGSBP (12 cyclic 2-layer windows) at I_max 25 on the same frames
    (the first timed step's channel seeds): both spend 50 M CN updates per frame at most (Sec. IV,
    equal check-update budget).  Per Eb/N0 point: FER, mean iterations, decode-only Gbit/s."""
    import numpy as np
    groups = nd.Groups.build(code, 12, 0.5, GROUP_SEED, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
    W = (c.N + 31) // 32
    llr = torch.empty((F, c.N), dtype=torch.float32, device=dev)
    hard = torch.empty((F, W), dtype=torch.int32, device=dev)
    out = {}
    for name, sched, imax in (("ndgsbp", nd.SCHEDULE_GROUPS, IMAX_ND), ("flooding", nd.SCHEDULE_FLOOD, IMAX_FLOOD)):
        p = nd.params_default(max_iter=imax, msg_dtype=nd.F32, schedule=sched)
        ws = torch.zeros(max(256, groups.workspace_size(p, F)), dtype=torch.uint8, device=dev)
        stats = torch.zeros((len(EBN0), nd.STATS_LEN), dtype=torch.int64, device=dev)
        nd.awgn_llr(code, F, EBN0[0], RATE, channel_seed(0, 0, rank), llr, stream=stream)
        nd.decode(groups, p, llr, ws, hard, stream=stream)   # warm-up
        ms = 0.0
        for i, eb in enumerate(EBN0):
            nd.awgn_llr(code, F, eb, RATE, channel_seed(i, 0, rank), llr, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nd.decode(groups, p, llr, ws, hard, stats=stats[i], stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        st = stats.cpu().numpy()
        fe = st[:, nd.STAT_FRAME_ERRORS]
        out[name] = {"max_iter": imax, "fer": (fe / F).tolist(),
                     "fer_ci95": [list(clopper_pearson(int(k), F)) for k in fe],
                     "mean_iterations": (st[:, nd.STAT_ITERATIONS] / F).tolist(),
                     "cn_updates_per_iter": int(c.M if sched == nd.SCHEDULE_FLOOD else groups.query()["cn_updates_per_iter"]),
                     "gbit_s": F * len(EBN0) * (c.N - c.M) / (ms / 1e3) / 1e9,
                     "plan": groups.plan(p, F).as_dict()["variant"]}
    out["what"] = (f"{F} frames per point, the same channel LLRs for both schedules; equal budget: NDGSBP "
                   f"{IMAX_ND} x {out['ndgsbp']['cn_updates_per_iter']} = flooding {IMAX_FLOOD} x {c.M} CN updates")
    return out


def precision_summary(nd, torch, dev, I, F):
    """FP32 / FP16 / BF16 message storage on the n=2304 r1/2 and n=16200 r2/3 codes at each code's
    FER ~ 1e-3 point: FER with its 95% Clopper-Pearson interval, decode-only Gbit/s (one timed
    launch after a warm-up), and FP16 / FP32 throughput."""
    out = {}
    st_ = torch.cuda.Stream(device=dev)
    for name in ("qc_n2304_r12", "qc_n16200_r23"):
        c, code, g = _setup_code(nd, I, name)
        eb = FER1E3_EBN0[name]
        W = (c.N + 31) // 32
        llr = torch.empty((F, c.N), dtype=torch.float32, device=dev)
        nd.awgn_llr(code, F, eb, I.design_rate(c), CHANNEL_SEED + c.N, llr, stream=st_)
        hard = torch.empty((F, W), dtype=torch.int32, device=dev)
        rows = {}
        for msg, dt in (("f32", nd.F32), ("f16", nd.F16), ("bf16", nd.BF16)):
            p = nd.params_default(max_iter=IMAX_ND, msg_dtype=dt)
            ws = torch.zeros(max(256, g.workspace_size(p, F)), dtype=torch.uint8, device=dev)
            stats = torch.zeros(nd.STATS_LEN, dtype=torch.int64, device=dev)
            nd.decode(g, p, llr, ws, hard, stream=st_)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st_)
            nd.decode(g, p, llr, ws, hard, stats=stats, stream=st_)
            e1.record(st_)
            torch.cuda.synchronize()
            s = stats.cpu().numpy()
            fe = int(s[nd.STAT_FRAME_ERRORS])
            rows[msg] = {"fer": fe / F, "fer_ci95": list(clopper_pearson(fe, F)),
                         "mean_iterations": float(s[nd.STAT_ITERATIONS] / F),
                         "gbit_s": F * (c.N - c.M) / (e0.elapsed_time(e1) / 1e3) / 1e9,
                         "variant": g.plan(p, F).variant}
            del ws
        rows["f16_over_f32"] = rows["f16"]["gbit_s"] / rows["f32"]["gbit_s"]
        rows["bf16_over_f32"] = rows["bf16"]["gbit_s"] / rows["f32"]["gbit_s"]
        rows["ebn0_db"] = eb
        out[name] = rows
        del llr
    out["what"] = f"{F} frames per code, the same LLRs for the three storage types, I_max {IMAX_ND}"
    return out


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
            seed = channel_seed(i, s, rank)
            nd.awgn_llr(code, F, eb, RATE, seed, llr, stream=stream)
            if timing is not None:
                timing.append(torch.cuda.Event(enable_timing=True))
                timing[-1].record(stream)
            stamp = latency and i == LATENCY_POINT
            nd.decode(groups, params, llr, ws, hard, iters, ok, stats=stats[i], iter_hist=hist,
                      start_ns=start_ns if stamp else None, retire_ns=retire_ns if stamp else None,
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
    elapsed_max = max_over_ranks(elapsed, dev, world)
    frames_total = F * len(EBN0) * args.steps * world
    value = whole_job_gbits(F * len(EBN0) * args.steps, world, 1152, elapsed_max)
    sum_over_ranks(stats, world)

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

    # roofline of the decode kernel: MUFU operations (3 per edge-update) over its launch time,
    # against the XU-pipe rate measured on this GPU for the kernel's 1:1:1 mix of ex2, rcp, lg2
    peaks, peak_kind = measured_peaks()
    dec_total_s = sum(dec_ms) / 1e3
    mufu_ops = MUFU_PER_EDGE_UPDATE * edge_updates_iter * iter_sum
    achieved = mufu_ops / dec_total_s / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    probe = mufu_peak(nd, torch, dev, sms, clk.get("sm_mhz") or peak_clock_mhz)
    peak = probe["mix_tops"]
    kname = {nd.VARIANT_QC: "qc_decode_kernel", nd.VARIANT_QC_GLOBAL: "qc_decode_kernel",
             nd.VARIANT_TILE: "tile_decode_kernel", nd.VARIANT_STREAM_SMEM: "stream_decode_kernel",
             nd.VARIANT_STREAM_GLOBAL: "stream_decode_kernel",
             nd.VARIANT_STREAM_BULK: "stream_decode_kernel"}.get(plan.variant, "decode_kernel")
    traffic, traffic_rec = profiled_traffic(kname)
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s", "frac": achieved / peak,
        "traffic": traffic,
        "what": f"MUFU ops (exp2+rcp+lg2 = {MUFU_PER_EDGE_UPDATE} per edge-update of Eq. (1)) of the decode "
                f"kernel over its CUDA-event time; peak = the XU-pipe rate of that 1:1:1 mix measured by "
                f"ndgsbp_mufu_probe on this GPU (per-op rates in mufu_probe); nominal "
                f"{MUFU_PER_CLK_PER_SM}/clk/SM x {sms} SMs x {peak_clock_mhz:.0f} MHz = "
                f"{MUFU_PER_CLK_PER_SM * sms * peak_clock_mhz * 1e6 / 1e12:.2f} Top/s",
        "mufu_probe": probe,
        "kernel": kname, "launches": len(dec_ms), "avg_launch_ms": sum(dec_ms) / len(dec_ms),
        "share_of_step": sum(dec_ms) / 1e3 / elapsed,
        "edge_updates_per_launch": edge_updates_iter * iter_sum / len(dec_ms),
        "hbm_bytes_per_launch_algorithmic": F * (c.N * 4 + W * 4 + 5),
        "hbm_frac_of_measured": F * (c.N * 4 + W * 4 + 5) / (sum(dec_ms) / len(dec_ms) / 1e3) / 1e9 / peaks["hbm_gbs"],
    }

    # beside the timed line: flooding at the same check-update budget (Sec. IV), and the message
    # precisions at each code's FER ~ 1e-3 point
    flood = None if args.no_extras else flood_equal_budget(nd, torch, dev, code, c, F, stream, rank)
    precision = None if args.no_extras else precision_summary(nd, torch, dev, I, args.extras_frames)

    # end-to-end through host buffers: pinned host LLRs -> device -> decode -> decisions back
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, nd, torch, code, c, groups, params, F, W, dev, rank, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        kept = []
        dt, nf, fe_or = oracle_sweep(args.cpu_frames, keep=kept)
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
        cpu["paired"] = paired_check(nd, torch, code, c, groups, params, kept, args.cpu_frames, dev, stream)
        # the same oracle on one core (a smaller sample)
        dt1, nf1, _ = oracle_sweep(args.cpu_frames_1core, threads=1)
        cpu["one_core"] = {"value": nf1 * 1152 / dt1 / 1e9, "unit": "Gbit/s", "cores": 1,
                           "sample": f"{args.cpu_frames_1core} frames at each of the {len(EBN0)} points, {dt1:.1f} s"}

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
                                f"(the {EBN0[LATENCY_POINT]} dB decode launch of the last timed step, the FER ~ 1e-3 "
                                f"point, {F} frames)"},
            "fer": fer, "ber": ber, "mean_iterations": iter_sum / max(frames_done, 1),
            "mean_iterations_per_point": (st[:, nd.STAT_ITERATIONS] / np.maximum(st[:, nd.STAT_FRAMES], 1)).tolist(),
            "coded_gbit_s": frames_total * c.N / elapsed_max / 1e9,
            "clocks": clk, "gpu_launches": 2 * len(EBN0) * args.steps,
            "plan": plan.as_dict(), "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
            "flooding_equal_budget": flood, "precision": precision,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_e2e(args, nd, torch, code, c, groups, params, F, W, dev, rank, world):
    """Same metric through the public API with host buffers: every step copies each point's
    LLRs from pinned host memory, decodes, and copies decisions, iteration counts and syndrome
    flags back.  Host-to-device copies, decodes and device-to-host copies run on three streams
    over two device buffers, so the next point's LLRs arrive while the current point decodes."""
    import numpy as np
    import torch.distributed as dist
    n_pts = len(EBN0)
    host_llr = []
    tmp = torch.empty((F, c.N), dtype=torch.float32, device=dev)
    for i, eb in enumerate(EBN0):
        nd.awgn_llr(code, F, eb, RATE, channel_seed(i, 0, rank, base=CHANNEL_SEED + 77), tmp)
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
    h2d_s = torch.cuda.Stream(device=dev)
    comp_s = torch.cuda.Stream(device=dev)
    d2h_s = torch.cuda.Stream(device=dev)
    # buffers alternate by a point counter that runs across steps; free[b] marks the end of the
    # device-to-host copies of the last point that used buffer b (its LLRs and outputs may then
    # be overwritten), so no copy overtakes a decode or a read-back of an earlier step
    ring = {"n": 0, "free": [None, None]}

    def one_step():
        for i in range(n_pts):
            b = ring["n"] % 2
            ring["n"] += 1
            with torch.cuda.stream(h2d_s):
                if ring["free"][b] is not None:
                    h2d_s.wait_event(ring["free"][b])
                d_llr[b].copy_(host_llr[i], non_blocking=True)
                loaded = torch.cuda.Event()
                loaded.record(h2d_s)
            with torch.cuda.stream(comp_s):
                comp_s.wait_event(loaded)
                nd.decode_plain(groups, params, d_llr[b], ws, d_hard[b], d_iters[b], d_ok[b], stream=comp_s)
                decoded = torch.cuda.Event()
                decoded.record(comp_s)
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(decoded)
                host_hard[i].copy_(d_hard[b], non_blocking=True)
                host_iters[i].copy_(d_iters[b], non_blocking=True)
                host_ok[i].copy_(d_ok[b], non_blocking=True)
                freed = torch.cuda.Event()
                freed.record(d2h_s)
            ring["free"][b] = freed

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
    dt = max_over_ranks(time.perf_counter() - t0, dev, world)
    frames = F * n_pts * args.steps * world
    h2d = n_pts * F * c.N * 4
    d2h = n_pts * F * (W * 4 + 4 + 1)
    ok_frac = float(host_ok.float().mean())
    # the read-back of the last point equals a device-resident decode of the same LLRs
    chk_llr = host_llr[n_pts - 1].to(dev)
    chk_hard = torch.empty((F, W), dtype=torch.int32, device=dev)
    chk_iters = torch.empty(F, dtype=torch.int32, device=dev)
    nd.decode_plain(groups, params, chk_llr, ws, chk_hard, chk_iters)
    torch.cuda.synchronize()
    match = bool(torch.equal(chk_hard.cpu(), host_hard[n_pts - 1]) and torch.equal(chk_iters.cpu(), host_iters[n_pts - 1]))
    return {"value": frames * 1152 / dt / 1e9, "unit": "Gbit/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * dt / args.steps,
            "timer": "host wall clock around all steps, synchronised", "syndrome_ok_fraction": ok_frac,
            "readback_matches_device_decode": match}


# ------------------------------------------------------------------------------------------
# supplementary workloads: ragged multi-code batches, serving, reduced-precision messages
# ------------------------------------------------------------------------------------------
# Eb/N0 of each code's FER ~ 1e-3 point (FP32 messages, cyclic 2-layer NDGSBP, I_max 25 for the
# n=2304 r1/2 and n=16200 codes, 30 for the others), interpolated between the two points of a
# GPU pre-sweep in 0.1 dB steps (262,144 frames per point, 131,072 for n=16200) that bracket
# FER = 1e-3: 2304 r1/2 1.7/1.8 dB (1.4e-3/5.4e-4), 16200 1.8/1.9 (4.6e-3/1.2e-4), 576
# 2.6/2.7 (1.2e-3/8.4e-4), 1152 2.7/2.8 (1.6e-3/8.2e-4), 2304 r3/4 2.8/2.9 (2.0e-3/6.4e-4),
# 8192 3.3/3.4 (1.3e-3/1.6e-4)
FER1E3_EBN0 = {"qc_n2304_r12": 1.75, "qc_n16200_r23": 1.85, "qc_n576_r12": 2.65, "qc_n1152_r23": 2.75,
               "qc_n2304_r34": 2.85, "qc_n8192_r2732": 3.3}
MIX4 = [("qc_n576_r12", 0.4), ("qc_n1152_r23", 0.3), ("qc_n2304_r34", 0.2), ("qc_n8192_r2732", 0.1)]
RAGGED_FRAMES = 200000


def _setup_code(nd, I, name, seed=2304):
    c = I.code_by_name(name)
    code = nd.Code.from_inputs(c)
    g = nd.Groups.build(code, c.M // c.Z, 0.5, seed, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
    return c, code, g


def _mufu_roofline(probe, mufu_ops, kernel_s, kernel, launches, extra=None):
    """MUFU roofline of a decode workload: mufu_ops (3 per edge-update, counted over the timed
    launches) over their CUDA-event time, against the measured rate of the 1:1:1 MUFU mix."""
    peak = probe["mix_tops"]
    achieved = mufu_ops / kernel_s / 1e12
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s", "frac": achieved / peak,
         "traffic": None, "kernel": kernel, "launches": launches, "avg_launch_ms": 1e3 * kernel_s / launches,
         "mufu_probe": probe,
         "what": "MUFU ops (3 per edge-update of Eq. (1)) over the kernels' CUDA-event time; peak = the measured "
                 "rate of the ex2/rcp/lg2 mix (ndgsbp_mufu_probe)"}
    if extra:
        r.update(extra)
    return r


def run_ragged(args):
    """Ragged batching over 200,000 frames of 4 QC codes in a 40/30/20/10 mix, FP16 messages,
    per-frame early stop, I_max 30, each code at its FER ~ 1e-3 point, replayed as a CUDA graph.
    The autotuner picks the launch: one persistent tile-kernel launch (block size, residency,
    per-code tile shape) or the per-code mode (each code's own plan, forked streams); the other
    mode is timed beside it.  A step = channel generation for the 4 codes + the ragged launch.
    Also beside it: the plain FP32 single-code batched path (each code's batch decoded by its own
    default launch, one after the other) on the same frames."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import inputs as I
    from paper_1202_1060_gb300 import ndgsbp as nd
    stream = torch.cuda.Stream(device=dev)
    batches = []
    for i, (name, share) in enumerate(MIX4):
        c, code, g = _setup_code(nd, I, name, seed=17 + i)
        F = int(RAGGED_FRAMES * share)
        W = (c.N + 31) // 32
        batches.append(dict(name=name, c=c, code=code, groups=g, F=F,
                            llr=torch.empty((F, c.N), dtype=torch.float32, device=dev),
                            hard_bits=torch.empty((F, W), dtype=torch.int32, device=dev),
                            iters=torch.empty(F, dtype=torch.int32, device=dev),
                            syndrome_ok=torch.empty(F, dtype=torch.uint8, device=dev),
                            stats=torch.zeros(nd.STATS_LEN, dtype=torch.int64, device=dev)))
    imax = 30

    def gen(s):
        for i, b in enumerate(batches):
            nd.awgn_llr(b["code"], b["F"], FER1E3_EBN0[b["name"]], I.design_rate(b["c"]),
                        CHANNEL_SEED + 31 * i + 1000 * s, b["llr"], stream=stream)

    gen(-1)
    torch.cuda.synchronize()
    p0 = nd.params_default(max_iter=imax, msg_dtype=nd.F16)
    t0 = time.perf_counter()
    params, tuned_ms = nd.ragged_autotune(batches, p0, sample_frames=8192,
                                          cache_path=os.path.join(OUT_DIR, "tune_cache.txt"))
    tune_s = time.perf_counter() - t0
    per_code_mode = params.variant == nd.VARIANT_RAGGED_PER_CODE
    # the other mode, timed on the same frames (tile: the library's default shape)
    other_p = nd.params_default(max_iter=imax, msg_dtype=nd.F16,
                                variant=nd.VARIANT_TILE if per_code_mode else nd.VARIANT_RAGGED_PER_CODE)
    other_b = [dict(b, frames_per_cta=0, lanes_per_cn=0) for b in batches] if per_code_mode else batches
    rg_other = nd.Ragged(other_b, other_p)
    for _ in range(2):
        rg_other.graph_launch(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        rg_other.graph_launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    other_ms = e0.elapsed_time(e1) / 3
    del rg_other
    rg = nd.Ragged(batches, params)
    plan, n_tiles = rg.info()
    for s in range(args.warmup):
        gen(-2 - s)
        rg.graph_launch(stream)
    torch.cuda.synchronize()
    for b in batches:
        b["stats"].zero_()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 2)]
    ev[0].record(stream)
    for s in range(args.steps):
        gen(s)
        ev[2 * s + 1].record(stream)
        rg.graph_launch(stream)
        ev[2 * s + 2].record(stream)
    ev[-1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = ev[0].elapsed_time(ev[-1]) / 1e3
    dec_s = sum(ev[2 * s + 1].elapsed_time(ev[2 * s + 2]) for s in range(args.steps)) / 1e3
    # a stats-carrying launch for FER and iterations (the graph replays the launch recorded at
    # create time, which carries the stats pointers)
    per_code = []
    bits = 0
    mufu = 0
    for b in batches:
        st = b["stats"].cpu().numpy()
        q = b["groups"].query()
        K = b["c"].N - b["c"].M
        bits += b["F"] * K
        mufu += MUFU_PER_EDGE_UPDATE * q["edge_updates_per_iter"] * int(st[nd.STAT_ITERATIONS])
        per_code.append({"code": b["name"], "frames": b["F"], "ebn0_db": FER1E3_EBN0[b["name"]],
                         "fer": float(st[nd.STAT_FRAME_ERRORS] / max(st[nd.STAT_FRAMES], 1)),
                         "mean_iterations": float(st[nd.STAT_ITERATIONS] / max(st[nd.STAT_FRAMES], 1)),
                         "frames_per_cta": b["frames_per_cta"], "lanes_per_cn": b["lanes_per_cn"]})
    value = bits * args.steps / elapsed / 1e9
    # plain FP32 single-code batched path on the same frames (last step's channel)
    pf = nd.params_default(max_iter=imax, msg_dtype=nd.F32)
    ws = [torch.zeros(max(256, b["groups"].workspace_size(pf, b["F"])), dtype=torch.uint8, device=dev)
          for b in batches]
    for _ in range(2):
        for b, w in zip(batches, ws):
            nd.decode_plain(b["groups"], pf, b["llr"], w, b["hard_bits"], b["iters"], b["syndrome_ok"], stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for b, w in zip(batches, ws):
        nd.decode_plain(b["groups"], pf, b["llr"], w, b["hard_bits"], b["iters"], b["syndrome_ok"], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_s = e0.elapsed_time(e1) / 1e3
    peaks, kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    line = {
        "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16", "data": "synthetic",
        "config": {"workload": "ragged: 200,000 frames of 4 QC codes (n=576 r1/2, 1152 r2/3, 2304 r3/4, 8192 r27/32) "
                               "in a 40/30/20/10 mix, FP16 messages, I_max 30, early stop, each code at its "
                               "FER~1e-3 Eb/N0, replayed as a CUDA graph; launch mode from the autotuner: "
                               + ("per-code plans on forked streams" if per_code_mode else
                                  "one persistent tile-kernel launch") + "; step = channel generation + decode",
                   "mode": "per_code" if per_code_mode else "tile",
                   "l2": "inputs larger than L2 (1.5 GB of LLRs)"},
        "decode_only_gbit_s": bits * args.steps / dec_s / 1e9,
        "plain_fp32_single_code_gbit_s": bits / plain_s / 1e9,
        "speedup_vs_plain_fp32": (bits * args.steps / dec_s) / (bits / plain_s),
        "per_code": per_code, "tuned": {"mode": "per_code" if per_code_mode else "tile",
                                        "block_threads": params.block_threads, "ctas_per_sm": params.ctas_per_sm,
                                        "launch_ms": tuned_ms, "tuning_s": tune_s, "tiles_or_codes": n_tiles,
                                        "plan": plan,
                                        "other_mode_ms": other_ms},
        "clocks": clk, "gpu_launches": (8 if per_code_mode else 5) * args.steps,
        # (mufu counts the timed launches: the replayed graph carries the statistics pointers)
        "roofline": _mufu_roofline(mufu_peak(nd, torch, dev, sms, clk.get("sm_mhz") or 2070.0), mufu, dec_s,
                                   "per-code launches (qc_decode_kernel for n=576/1152/2304, stream_decode_kernel "
                                   "for n=8192) on forked streams" if per_code_mode else "tile_decode_kernel",
                                   args.steps),
        "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Serving: Poisson arrivals of decode requests (sizes log-uniform in [1, 4096] frames, code
    by the 40/30/20/10 mix, Eb/N0 ~ U[1, 3] dB, I_max 30, FP16 messages) at 0.5, 0.75, 1.0 and
    1.2x the server's saturated capacity; latency = completion - scheduled arrival."""
    import numpy as np
    import torch
    import threading
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import inputs as I
    from paper_1202_1060_gb300 import ndgsbp as nd
    rng = np.random.default_rng(args.arrival_seed)
    grid = [1.0 + 0.25 * i for i in range(9)]
    pool_frames = 4096
    codes = []
    for i, (name, share) in enumerate(MIX4):
        c, code, g = _setup_code(nd, I, name, seed=17 + i)
        tmp = torch.empty((pool_frames, c.N), dtype=torch.float32, device=dev)
        pools = []
        for j, eb in enumerate(grid):
            nd.awgn_llr(code, pool_frames, eb, I.design_rate(c), CHANNEL_SEED + 7919 * i + j, tmp)
            pools.append(tmp.cpu().numpy().copy())
        codes.append(dict(name=name, c=c, code=code, groups=g, share=share, pools=pools, K=c.N - c.M))
    del tmp
    params = nd.params_default(max_iter=30, msg_dtype=nd.F16)
    budget = args.serve_budget_mb << 20
    srv = nd.Server([d["groups"] for d in codes], params, budget, epoch_iters=args.epoch_iters,
                    weights=[d["share"] * d["c"].N for d in codes])

    def draw_request():
        k = int(rng.choice(len(codes), p=[d["share"] for d in codes]))
        size = int(np.clip(np.floor(np.exp(rng.uniform(0.0, np.log(4097.0)))), 1, 4096))
        eb = rng.uniform(1.0, 3.0)
        j = int(np.argmin([abs(eb - x) for x in grid]))
        off = int(rng.integers(0, pool_frames - size + 1))
        return k, codes[k]["pools"][j][off:off + size]

    # capacity: a saturated backlog
    backlog = [draw_request() for _ in range(args.serve_backlog)]
    for k, llr in backlog[:32]:
        srv.submit(k, llr).wait(600000)
    st_a = srv.stats()
    t0 = time.perf_counter()
    reqs = [srv.submit(k, llr) for k, llr in backlog]
    for r in reqs:
        r.wait(600000)
    cap_s = time.perf_counter() - t0
    st_b = srv.stats()
    cap_split = {k: st_b[k] - st_a[k] for k in ("epochs", "admit_seconds", "device_seconds", "harvest_seconds",
                                                "busy_seconds", "iterations", "frames_completed")}
    cap_frames = sum(llr.shape[0] for _, llr in backlog)
    cap_bits = sum(llr.shape[0] * codes[k]["K"] for k, llr in backlog)
    capacity = cap_frames / cap_s
    mean_size = cap_frames / len(backlog)
    loads = []
    clocks = ClockSampler(0)
    clocks.start()
    for load in (0.5, 0.75, 1.0, 1.2):
        rate = load * capacity / mean_size          # requests per second
        n_req = max(50, int(rate * args.serve_seconds))
        gaps = rng.exponential(1.0 / rate, n_req)
        arrivals = np.cumsum(gaps)
        work = [draw_request() for _ in range(n_req)]
        handles = [None] * n_req
        st0 = srv.stats()
        start = time.perf_counter()
        for i in range(n_req):
            now = time.perf_counter() - start
            if arrivals[i] > now:
                time.sleep(arrivals[i] - now)
            handles[i] = srv.submit(work[i][0], work[i][1])
        for h in handles:
            h.wait(600000)
        end = time.perf_counter() - start
        # latency from the scheduled arrival: submit lateness (client behind schedule) counts
        lat = []
        for i, h in enumerate(handles):
            lat.append(h.latency_ms)
        st1 = srv.stats()
        frames = sum(w[1].shape[0] for w in work)
        bits = sum(w[1].shape[0] * codes[w[0]]["K"] for w in work)
        loads.append({"load": load, "requests": n_req, "frames": frames, "offered_frames_per_s": load * capacity,
                      "seconds": end, "gbit_s": bits / end / 1e9,
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "epochs": st1["epochs"] - st0["epochs"],
                      "frame_errors_unsatisfied": st1["frame_errors_unsatisfied"] - st0["frame_errors_unsatisfied"],
                      "mean_iterations": (st1["iterations"] - st0["iterations"]) / max(frames, 1)})
    clk = clocks.stop()
    stats = srv.stats()
    srv.close()
    # the plain batched path on the same frames: each code's frames of the backlog in one
    # device-resident batch, decoded by the default single-code launch (FP32 and FP16 messages)
    plain = {}
    for mname, mdt in (("f32", nd.F32), ("f16", nd.F16)):
        pp = nd.params_default(max_iter=30, msg_dtype=mdt)
        jobs = []
        for k, d in enumerate(codes):
            frames = [llr for kk, llr in backlog if kk == k]
            if not frames:
                continue
            x = torch.from_numpy(np.concatenate(frames)).to(dev)
            F = x.shape[0]
            W = (d["c"].N + 31) // 32
            jobs.append((d, x, torch.zeros(max(256, d["groups"].workspace_size(pp, F)), dtype=torch.uint8, device=dev),
                         torch.empty((F, W), dtype=torch.int32, device=dev)))
        for _ in range(2):
            for d, x, w, hb in jobs:
                nd.decode_plain(d["groups"], pp, x, w, hb)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for d, x, w, hb in jobs:
            nd.decode_plain(d["groups"], pp, x, w, hb)
        e1.record()
        torch.cuda.synchronize()
        plain[mname] = cap_bits / (e0.elapsed_time(e1) / 1e3) / 1e9
        del jobs
    sat = {"frames_per_s": capacity, "gbit_s": cap_bits / cap_s / 1e9, "requests": len(backlog),
           "seconds": cap_s, "server_time_split": cap_split,
           "plain_batched_gbit_s": plain,
           "what": "saturated backlog through the server (host buffers in and out) vs the same frames decoded "
                   "as device-resident per-code batches by the default single-code launch"}
    line = {
        "metric": METRIC, "value": sat["gbit_s"], "unit": "Gbit/s", "n_gpus": 1, "steps": len(loads),
        "warmup": 32, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16", "data": "synthetic",
        "config": {"workload": "serving: Poisson arrivals at 0.5/0.75/1.0/1.2x saturated capacity, request sizes "
                               "log-uniform in [1, 4096] frames, codes by the 40/30/20/10 mix of n=576/1152/2304/8192, "
                               "Eb/N0 ~ U[1,3] dB (nearest 0.25 dB pool), FP16 messages, I_max 30, continuous "
                               "batching with device-resident frame state; per epoch one serving launch per pool of the "
                               "kernel its plain decode uses (the layered QC kernel for n=576/1152/2304, the "
                               "stream kernel for n=8192), forked",
                   "hbm_budget_mb": args.serve_budget_mb, "epoch_iters": args.epoch_iters,
                   "arrival_seed": args.arrival_seed, "slots": stats["slots_total"],
                   "l2": "pool state larger than L2"},
        "saturated": sat, "loads": loads, "clocks": clk, "gpu_launches": stats["launches"],
        "latency": {"p50_ms": loads[2]["p50_ms"], "p99_ms": loads[2]["p99_ms"],
                    "what": "request completion - submission at 1.0x capacity (host clock)"},
        "roofline": None, "e2e": {"value": sat["gbit_s"], "unit": "Gbit/s",
                                  "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                                  "what": "host buffers in and out through the server API"},
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


EDGE_ERR_FRAMES = 64
EDGE_ERR_ITERS = (1, 5)


def edge_error(nd, torch, g, msg_dtype, llr, ref_k, stream):
    """Largest per-edge CN->VN message error of the GPU against the oracle's (ref_k[k], natural
    LLR units) after k iterations without early stop, on the frames of llr: absolute and relative
    to max(|L_oracle|, 1)."""
    import numpy as np
    dev = llr.device
    F, E = llr.shape[0], int(ref_k[EDGE_ERR_ITERS[0]].shape[1])
    W = (llr.shape[1] + 31) // 32
    hard = torch.empty((F, W), dtype=torch.int32, device=dev)
    msgs = torch.zeros((F, E), dtype=torch.float32, device=dev)
    out = {"frames": F}
    for k in EDGE_ERR_ITERS:
        p = nd.params_default(max_iter=k, msg_dtype=msg_dtype, early_stop=0)
        ws = torch.zeros(max(256, g.workspace_size(p, F)), dtype=torch.uint8, device=dev)
        nd.decode(g, p, llr, ws, hard, messages=msgs, stream=stream)
        torch.cuda.synchronize()
        m, r = msgs.cpu().numpy(), ref_k[k]
        d = np.abs(m - r)
        out[f"k{k}"] = {"max_abs": float(d.max()), "max_rel": float((d / np.maximum(np.abs(r), 1.0)).max())}
    return out


def run_precision(args):
    """Reduced-precision messages: the n=2304 r1/2 and n=16200 r2/3 QC codes at their FER ~ 1e-3
    points, 262,144 frames, FP32 / FP16 / BF16 message storage with FP32 arithmetic.  The FP64
    oracle decodes the first --precision-oracle-frames (n=2304) and a quarter of that (n=16200) of
    the same LLRs: every storage type's FER on those frames must lie inside the oracle's 95%
    Clopper-Pearson interval, and so must its FER over all frames.  Each row also states the
    largest per-edge message error against the oracle after 1 and 5 iterations on 64 frames."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__
    __graft_entry__.build_library()
    from oracle import oracle as O
    from paper_1202_1060_gb300 import inputs as I
    from paper_1202_1060_gb300 import ndgsbp as nd
    O.build()
    stream = torch.cuda.Stream(device=dev)
    F = args.precision_frames
    rows, oracle_rows = [], []
    clocks = ClockSampler(0)
    clocks.start()
    mufu_total = {}
    for name in ("qc_n2304_r12", "qc_n16200_r23"):
        c, code, g = _setup_code(nd, I, name)
        eb = FER1E3_EBN0[name]
        llr = torch.empty((F, c.N), dtype=torch.float32, device=dev)
        nd.awgn_llr(code, F, eb, I.design_rate(c), CHANNEL_SEED + c.N, llr, stream=stream)
        W = (c.N + 31) // 32
        hard = torch.empty((F, W), dtype=torch.int32, device=dev)
        iters = torch.empty(F, dtype=torch.int32, device=dev)
        ok = torch.empty(F, dtype=torch.uint8, device=dev)
        stats = torch.zeros(nd.STATS_LEN, dtype=torch.int64, device=dev)
        q = g.query()
        n_or = args.precision_oracle_frames if c.N <= 2304 else args.precision_oracle_frames // 4
        n_or = min(n_or, F)
        # the oracle on the first n_or frames of the same LLRs (FP64 of the FP32 values)
        torch.cuda.synchronize()
        host = llr[:n_or].cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        ref = O.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], host, IMAX_ND, want_total=False)
        t_or = time.perf_counter() - t0
        del host
        fe_or = int(ref.hard.any(axis=1).sum())
        lo, hi = clopper_pearson(fe_or, n_or)
        oracle_rows.append({"code": name, "frames": n_or, "fer": fe_or / n_or, "fer_ci95": [lo, hi],
                            "seconds": t_or, "frames_per_s": n_or / t_or, "gbit_s": n_or * (c.N - c.M) / t_or / 1e9,
                            "cores": host_cores()})
        # per-edge message error: the oracle's CN->VN messages after k iterations (no early stop)
        # of the first EDGE_ERR_FRAMES frames
        n_e = min(EDGE_ERR_FRAMES, F)
        host_e = llr[:n_e].cpu().numpy().astype(np.float64)
        ref_k = {k: O.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], host_e, k, early_stop=False, want_total=False,
                                    want_c2v=True).c2v for k in EDGE_ERR_ITERS}
        del host_e
        for msg, dt in (("f32", nd.F32), ("f16", nd.F16), ("bf16", nd.BF16)):
            p = nd.params_default(max_iter=IMAX_ND, msg_dtype=dt)
            ws = torch.zeros(max(256, g.workspace_size(p, F)), dtype=torch.uint8, device=dev)
            for _ in range(args.warmup):
                nd.decode(g, p, llr, ws, hard, iters, ok, stream=stream)
            stats.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                nd.decode(g, p, llr, ws, hard, iters, ok, stats=stats, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            st = stats.cpu().numpy()
            plan = g.plan(p, F)
            # FER of this storage type on the oracle's frames (the last decode's outputs)
            bits = nd.unpack_bits(hard[:n_or], c.N)
            fe_pair = int(bits.any(axis=1).sum())
            fer_all = float(st[nd.STAT_FRAME_ERRORS] / st[nd.STAT_FRAMES])
            mufu = MUFU_PER_EDGE_UPDATE * q["edge_updates_per_iter"] * float(st[nd.STAT_ITERATIONS])
            mufu_total[(name, msg)] = (mufu, sec)
            rows.append({"code": name, "msg_dtype": msg, "ebn0_db": eb, "frames": F,
                         "gbit_s": F * args.steps * (c.N - c.M) / sec / 1e9,
                         "fer": fer_all, "fer_ci95": list(clopper_pearson(int(st[nd.STAT_FRAME_ERRORS] / args.steps), F)),
                         "fer_on_oracle_frames": fe_pair / n_or,
                         "inside_oracle_ci": bool(lo <= fe_pair / n_or <= hi and lo <= fer_all <= hi),
                         "ber": float(st[nd.STAT_BIT_ERRORS] / (st[nd.STAT_FRAMES] * c.N)),
                         "mean_iterations": float(st[nd.STAT_ITERATIONS] / st[nd.STAT_FRAMES]),
                         "variant": plan.variant, "ms_per_decode": 1e3 * sec / args.steps,
                         "mufu_tops": mufu / sec / 1e12,
                         "max_edge_error": edge_error(nd, torch, g, dt, llr[:n_e], ref_k, stream)})
            del ws
        del llr
    clk = clocks.stop()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    probe = mufu_peak(nd, torch, dev, sms, clk.get("sm_mhz") or 2070.0)
    f16 = [r for r in rows if r["msg_dtype"] == "f16"]
    big = mufu_total[("qc_n16200_r23", "f16")]
    for r in rows:
        r["mufu_frac"] = r["mufu_tops"] / probe["mix_tops"]
    t_or = sum(o["seconds"] for o in oracle_rows)
    line = {
        "metric": METRIC, "value": sum(r["gbit_s"] for r in f16) / len(f16), "unit": "Gbit/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": f"precision: n=2304 r1/2 and n=16200 r2/3 QC codes at FER~1e-3, {F} frames, "
                               "cyclic 2-layer NDGSBP, I_max 25, FP32/FP16/BF16 message storage",
                   "l2": "inputs larger than L2"},
        "rows": rows, "oracle": oracle_rows,
        "f16_over_f32": {n: next(r["gbit_s"] for r in rows if r["code"] == n and r["msg_dtype"] == "f16") /
                         next(r["gbit_s"] for r in rows if r["code"] == n and r["msg_dtype"] == "f32")
                         for n in ("qc_n2304_r12", "qc_n16200_r23")},
        "all_inside_oracle_ci": all(r["inside_oracle_ci"] for r in rows),
        "clocks": clk, "gpu_launches": 6 * (args.steps + args.warmup),
        "roofline": _mufu_roofline(probe, big[0], big[1], "stream_decode_kernel (n=16200, FP16)", args.steps),
        "e2e": None,
        "cpu_baseline": {"value": sum(o["frames"] * 1.0 for o in oracle_rows) / t_or, "unit": "frames/s",
                         "cores": host_cores(), "kind": "oracle",
                         "sample": "; ".join(f"{o['frames']} frames of {o['code']}" for o in oracle_rows)},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_decode(args):
    """One code alone (the profiling command of the committed kernel summaries): --code at --ebn0,
    --frames frames of GPU-generated LLRs, cyclic 2-layer NDGSBP (or --vertical G VN groups),
    I_max 25, --msg storage, --variant; --warmup untimed then --steps timed decodes (CUDA events).
    Beside it: the MUFU roofline of the schedule's Eq. (1) operations against the per-op rates
    measured by ndgsbp_mufu_probe, and the FP64 oracle (same schedule and groups) timed on the
    host cores on the first --decode-oracle-frames frames, with the frames on which GPU and
    oracle disagree about a frame error counted."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import inputs as I
    from paper_1202_1060_gb300 import ndgsbp as nd
    c, code, g = _setup_code(nd, I, args.code)
    F = args.frames
    eb = args.ebn0 if args.ebn0 is not None else FER1E3_EBN0.get(args.code, 2.0)
    st_ = torch.cuda.Stream(device=dev)
    llr = torch.empty((F, c.N), dtype=torch.float32, device=dev)
    nd.awgn_llr(code, F, eb, I.design_rate(c), CHANNEL_SEED + c.N, llr, stream=st_)
    W = (c.N + 31) // 32
    hard = torch.empty((F, W), dtype=torch.int32, device=dev)
    stats = torch.zeros(nd.STATS_LEN, dtype=torch.int64, device=dev)
    dt = {"f32": nd.F32, "f16": nd.F16, "bf16": nd.BF16}[args.msg]
    p = nd.params_default(max_iter=IMAX_ND, msg_dtype=dt, variant=args.variant, ctas_per_sm=args.ctas_per_sm)
    from oracle import oracle as O
    O.build()
    q = g.query()
    deg = np.diff(np.asarray(c.row_ptr, dtype=np.int64))
    if args.vertical > 0:
        # the vertical (VN-group) schedule with --vertical random VN groups
        vg = nd.VGroups.build(code, args.vertical, GROUP_SEED)
        vq = vg.query()
        oracle_run = lambda x: O.vertical_decode(c, vq["grp_ptr"], vq["grp_vn"], x, IMAX_ND, want_total=False)
        # Eq. (1) per edge of a group's VNs: d - 1 exponentials, one reciprocal and one logarithm
        ops_per_iter = {"ex2": int((deg * (deg - 1)).sum()), "rcp": int(c.E), "lg2": int(c.E)}
        sched = f"vertical shuffled BP, {args.vertical} VN groups"
        ws = torch.zeros(max(256, vg.workspace_size(p, F)), dtype=torch.uint8, device=dev)
        run = lambda **kw: nd.decode_vertical(vg, p, llr, ws, hard, stream=st_, **kw)
        plan = {"schedule": "vertical", "G": args.vertical, "workspace_bytes": vg.workspace_size(p, F)}
    else:
        sched = "cyclic 2-layer NDGSBP"
        oracle_run = lambda x: O.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], x, IMAX_ND, want_total=False)
        eu = q["edge_updates_per_iter"]
        ops_per_iter = {"ex2": eu, "rcp": eu, "lg2": eu}
        ws = torch.zeros(max(256, g.workspace_size(p, F)), dtype=torch.uint8, device=dev)
        run = lambda **kw: nd.decode(g, p, llr, ws, hard, stream=st_, **kw)
        plan = g.plan(p, F).as_dict()
    for _ in range(args.warmup):
        run()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st_)
    for _ in range(args.steps):
        run(stats=stats)
    e1.record(st_)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = e0.elapsed_time(e1) / 1e3
    s = stats.cpu().numpy()
    # MUFU roofline: the schedule's operations at the measured per-op rates
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    probe = mufu_peak(nd, torch, dev, sms, clk.get("sm_mhz") or 2070.0)
    iters_total = float(s[nd.STAT_ITERATIONS])
    n_ops = {k: v * iters_total for k, v in ops_per_iter.items()}
    t_mufu = sum(n_ops[k] / (probe[k]["tops"] * 1e12) for k in n_ops)
    ops = sum(n_ops.values())
    roof = {"bound": "alu", "achieved": ops / sec / 1e12, "peak": ops / t_mufu / 1e12, "unit": "Top/s",
            "frac": t_mufu / sec, "traffic": None, "mufu_ops": {k: int(v) for k, v in n_ops.items()},
            "mufu_probe": probe,
            "what": "Eq. (1)'s ex2/rcp/lg2 operations of the timed decodes over their CUDA-event time; peak = the "
                    "rate of this operation mix at the per-op rates measured by ndgsbp_mufu_probe"}
    # the oracle beside it, on the first frames of the same LLRs; paired frame-error status
    n_or = min(args.decode_oracle_frames if args.decode_oracle_frames > 0 else (256 if c.N <= 2304 else 64), F)
    host = llr[:n_or].cpu().numpy().astype(np.float64)
    t0 = time.perf_counter()
    ref = oracle_run(host)
    t_or = time.perf_counter() - t0
    run()   # the GPU's decisions on all frames (no statistics)
    torch.cuda.synchronize()
    bits = nd.unpack_bits(hard[:n_or], c.N)
    cpu = {"value": n_or * (c.N - c.M) / t_or / 1e9, "unit": "Gbit/s", "cores": host_cores(), "kind": "oracle",
           "sample": f"the first {n_or} of the {F} frames, same schedule and groups, {t_or:.1f} s",
           "frames_per_s": n_or / t_or,
           "frame_error_status_differs": int((bits.any(axis=1) != ref.hard.any(axis=1)).sum()),
           "oracle_frame_errors": int(ref.hard.any(axis=1).sum())}
    line = {"metric": METRIC, "value": F * args.steps * (c.N - c.M) / sec / 1e9, "unit": "Gbit/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.msg, "data": "synthetic",
            "config": {"workload": f"decode: {args.code} at {eb} dB, {F} frames, {sched}, I_max {IMAX_ND}"},
            "fer": float(s[nd.STAT_FRAME_ERRORS] / max(s[nd.STAT_FRAMES], 1)),
            "mean_iterations": float(s[nd.STAT_ITERATIONS] / max(s[nd.STAT_FRAMES], 1)),
            "plan": plan, "clocks": clk, "gpu_launches": args.steps, "roofline": roof, "e2e": None,
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


GA_ENSEMBLES = [("(3,6)", {3: 1.0}, {6: 1.0}, 0.5, 1.163), ("(4,6)", {4: 1.0}, {6: 1.0}, 1 / 3, 1.730)]
GA_SCHEDULES = [("flooding", 1, 0.0), ("GSBP", 4, 0.0), ("NDGSBP", 4, 0.4)]


def run_ga(args):
    """The Gaussian-approximation analysis of Sec. III in FP64 on the GPU beside the oracle's
    (oracle/ga.py), closed-form Phi (the form that reproduces Table I): per ensemble and schedule,
    the threshold to 1e-4 dB (the library's grid bracketing, the oracle's bisection) and the
    iterations to error-free decoding 0.05 dB above the printed flooding threshold; and a batch of
    1,024 Eb/N0 points (0.5-3 dB) run through the recursion in one launch per schedule, timed
    against the oracle on 32 of those points."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build_library()
    from oracle import ga
    from paper_1202_1060_gb300 import ndgsbp as nd
    pk = nd.GA_PHI_CLOSED

    def gpu_run(lam, rho, R, G, r, snr):
        if G == 1:
            return nd.ga_flood(lam, rho, R, snr, phi_kind=pk)
        return nd.ga_groups(lam, rho, R, G, r, snr, phi_kind=pk)

    def gpu_threshold(lam, rho, R, G, r):
        if G == 1:
            return nd.ga_flood_threshold(lam, rho, R, phi_kind=pk, lo_db=0.5, hi_db=3.0, tol_db=1e-4)
        return nd.ga_groups_threshold(lam, rho, R, G, r, phi_kind=pk, lo_db=0.5, hi_db=3.0, tol_db=1e-4)

    def oracle_run(lam, rho, R, G, r, e):
        if G == 1:
            return ga.flood_ga(e, lam, rho, R, kind="approx")
        return ga.group_ga(e, lam, rho, R, G, r, kind="approx")

    rows = []
    snr = np.linspace(0.5, 3.0, 1024)
    sample = snr[::32]
    gpu_points_s, or_points_s, agree, total = 0.0, 0.0, 0, 0
    for name, lam, rho, R, printed in GA_ENSEMBLES:
        for sched, G, r in GA_SCHEDULES:
            t0 = time.perf_counter()
            th_gpu = gpu_threshold(lam, rho, R, G, r)
            t_th_gpu = time.perf_counter() - t0
            t0 = time.perf_counter()
            th_or = ga.threshold(lambda e: oracle_run(lam, rho, R, G, r, e), lo=0.5, hi=3.0, tol=1e-4)
            t_th_or = time.perf_counter() - t0
            _, it_gpu, _ = gpu_run(lam, rho, R, G, r, np.array([printed + 0.05]))
            _, it_or, _ = oracle_run(lam, rho, R, G, r, printed + 0.05)
            gpu_run(lam, rho, R, G, r, snr)   # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cv, it, _ = gpu_run(lam, rho, R, G, r, snr)
            t_b_gpu = time.perf_counter() - t0
            t0 = time.perf_counter()
            ref = [oracle_run(lam, rho, R, G, r, float(e)) for e in sample]
            t_b_or = time.perf_counter() - t0
            same = sum(int(bool(cv[32 * k]) == bool(ref[k][0])) for k in range(len(sample)))
            agree += same
            total += len(sample)
            gpu_points_s += len(snr) / t_b_gpu
            or_points_s += len(sample) / t_b_or
            rows.append({"ensemble": name, "schedule": sched, "G": G, "r": r,
                         "threshold_db": {"gpu": th_gpu, "oracle": th_or, "table_I_flooding": printed},
                         "threshold_seconds": {"gpu": t_th_gpu, "oracle": t_th_or},
                         "iterations_at_threshold_plus_0.05dB": {"gpu": int(it_gpu[0]), "oracle": int(it_or)},
                         "batch": {"points": len(snr), "gpu_seconds": t_b_gpu, "gpu_points_per_s": len(snr) / t_b_gpu,
                                   "oracle_points": len(sample), "oracle_seconds": t_b_or,
                                   "oracle_points_per_s": len(sample) / t_b_or,
                                   "convergence_agrees_on_oracle_points": f"{same}/{len(sample)}"}})
    n = len(rows)
    line = {"metric": "GA recursion Eb/N0 points per second (FP64)", "value": gpu_points_s / n,
            "unit": "points/s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "GA analysis (Sec. III, Eqs. (4)-(17)): (3,6) and (4,6) ensembles; flooding, GSBP "
                                   "(4 groups), NDGSBP (4 groups, r = 0.4); closed-form Phi; 1,024 Eb/N0 points"},
            "rows": rows, "convergence_agreement": f"{agree}/{total}",
            "roofline": None, "e2e": None,
            "cpu_baseline": {"value": or_points_s / n, "unit": "points/s", "cores": 1, "kind": "oracle",
                             "sample": "32 of the 1,024 points per ensemble and schedule, oracle/ga.py on one core"}}
    print(json.dumps(line), flush=True)
    return 0


def run_c1(args):
    """The Gallager (3,6) n=1008 workload: 500 frames at Eb/N0 1.5 dB, FP64 channel LLRs, flooding,
    disjoint GSBP (4 groups) and NDGSBP (4 groups, r = 0.4) at I_max 50, and NDGSBP at the equal
    check-update budget I_ND = floor(50 M / U) = 35 (Sec. IV).  GPU and FP64 oracle decode the same
    LLRs; per schedule: FER and BER with the oracle's 95% interval, mean iterations, and GPU
    throughput (the 500 frames, and 65,536 frames of the same kind)."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__
    __graft_entry__.build_library()
    from oracle import oracle as O
    from paper_1202_1060_gb300 import inputs as I
    from paper_1202_1060_gb300 import ndgsbp as nd
    O.build()
    c = I.code_by_name("gallager36_n1008")
    code = nd.Code.from_inputs(c)
    F, eb = 500, 1.5
    host = I.channel_llr(c.N, F, eb, 0.5, seed=1008)
    big_F = 65536
    big = torch.empty((big_F, c.N), dtype=torch.float32, device=dev)
    nd.awgn_llr(code, big_F, eb, 0.5, CHANNEL_SEED + 1008, big)
    d_llr = torch.from_numpy(host).to(dev)
    W = (c.N + 31) // 32
    schedules = [("flooding", 1, 0.0, nd.SCHEDULE_FLOOD, 50), ("gsbp", 4, 0.0, nd.SCHEDULE_GROUPS, 50),
                 ("ndgsbp", 4, 0.4, nd.SCHEDULE_GROUPS, 50), ("ndgsbp_equal_budget", 4, 0.4, nd.SCHEDULE_GROUPS, None)]
    rows = []
    for name, G, r, sched, imax in schedules:
        g = nd.Groups.build(code, G, r, 7)
        qq = g.query()
        if imax is None:
            imax = int(50 * c.M // qq["cn_updates_per_iter"])
        p = nd.params_default(max_iter=imax, schedule=sched)
        out = {}
        for tag, llr, n in (("c1", d_llr, F), ("large", big, big_F)):
            ws = torch.zeros(max(256, g.workspace_size(p, n)), dtype=torch.uint8, device=dev)
            hard = torch.empty((n, W), dtype=torch.int32, device=dev)
            stats = torch.zeros(nd.STATS_LEN, dtype=torch.int64, device=dev)
            for _ in range(args.warmup):
                nd.decode(g, p, llr, ws, hard)
            stats.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                nd.decode(g, p, llr, ws, hard, stats=stats)
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            st = stats.cpu().numpy() / args.steps
            out[tag] = {"frames": n, "gbit_s": n * args.steps * (c.N - c.M) / sec / 1e9, "fer": float(st[nd.STAT_FRAME_ERRORS] / n),
                        "ber": float(st[nd.STAT_BIT_ERRORS] / (n * c.N)), "mean_iterations": float(st[nd.STAT_ITERATIONS] / n),
                        "variant": g.plan(p, n).variant}
        # the oracle on the same 500 frames
        t0 = time.perf_counter()
        if sched == nd.SCHEDULE_FLOOD:
            ref = O.flood_decode(c, host, imax, want_total=False)
        else:
            ref = O.ndgsbp_decode(c, qq["grp_ptr"], qq["cn_idx"], host, imax, want_total=False)
        t_or = time.perf_counter() - t0
        fe, be = int(ref.hard.any(axis=1).sum()), int(ref.hard.sum())
        lo, hi = clopper_pearson(fe, F)
        blo, bhi = clopper_pearson(be, F * c.N)
        gpu = out["c1"]
        rows.append({"schedule": name, "groups": G, "r": r, "max_iter": imax,
                     "cn_updates_per_iter": int(c.M if sched == nd.SCHEDULE_FLOOD else qq["cn_updates_per_iter"]),
                     "gpu": gpu, "gpu_65536_frames": out["large"],
                     "oracle": {"fer": fe / F, "fer_ci95": [lo, hi], "ber": be / (F * c.N), "ber_ci95": [blo, bhi],
                                "mean_iterations": float(ref.iters.mean()), "seconds": t_or},
                     "gpu_inside_oracle_ci": bool(lo <= gpu["fer"] <= hi and blo <= gpu["ber"] <= bhi)})
    t_or = sum(rw["oracle"]["seconds"] for rw in rows)
    line = {
        "metric": METRIC, "value": next(rw["gpu_65536_frames"]["gbit_s"] for rw in rows if rw["schedule"] == "ndgsbp"),
        "unit": "Gbit/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "Gallager (3,6) n=1008 (seeded, 4-cycle-free), Eb/N0 1.5 dB, 500 frames, FP64 channel "
                               "LLRs; flooding, GSBP (4 groups), NDGSBP (4 groups, r = 0.4) at I_max 50 and NDGSBP "
                               "at the equal check-update budget; value = NDGSBP on 65,536 such frames"},
        "rows": rows, "all_inside_oracle_ci": all(rw["gpu_inside_oracle_ci"] for rw in rows),
        "roofline": None, "e2e": None,
        "cpu_baseline": {"value": 4 * F * (c.N - c.M) / t_or / 1e9, "unit": "Gbit/s", "cores": host_cores(),
                         "kind": "oracle", "sample": f"the same {F} frames under the 4 schedules, {t_or:.2f} s"},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=FRAMES, help="frames per Eb/N0 point per GPU")
    ap.add_argument("--variant", type=int, default=0, help="decode variant (0 = library choice)")
    ap.add_argument("--cpu-frames", type=int, default=4096, help="oracle sample per Eb/N0 point")
    ap.add_argument("--cpu-frames-1core", type=int, default=64, help="one-core oracle sample per Eb/N0 point")
    ap.add_argument("--ref-frames", type=int, default=64, help="oracle frames per point per reference step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the flooding and precision extras")
    ap.add_argument("--extras-frames", type=int, default=65536, help="frames per code and dtype, precision extra")
    ap.add_argument("--workload", choices=["sweep", "ragged", "serving", "precision", "c1", "decode", "ga"],
                    default="sweep",
                    help="sweep = the default n=2304 Eb/N0 sweep line; the others are supplementary")
    ap.add_argument("--precision-frames", type=int, default=262144)
    ap.add_argument("--code", default="qc_n16200_r23", help="decode workload: the code")
    ap.add_argument("--ebn0", type=float, default=None, help="decode workload: Eb/N0 (default: the FER~1e-3 point)")
    ap.add_argument("--msg", choices=["f32", "f16", "bf16"], default="f16", help="decode workload: message storage")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="decode workload: residency cap (0 = library choice)")
    ap.add_argument("--decode-oracle-frames", type=int, default=0,
                    help="decode workload: frames the oracle decodes beside it (0 = 256 up to n=2304, else 64)")
    ap.add_argument("--vertical", type=int, default=0,
                    help="decode workload: decode with the vertical schedule over this many VN groups (0 = NDGSBP)")
    ap.add_argument("--precision-oracle-frames", type=int, default=65536,
                    help="oracle frames for n=2304 (a quarter of that for n=16200)")
    ap.add_argument("--serve-budget-mb", type=int, default=2048)
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-backlog", type=int, default=10500,
                    help="requests of the saturated capacity window (about 3 s of work)")
    ap.add_argument("--epoch-iters", type=int, default=30)
    ap.add_argument("--arrival-seed", type=int, default=20260)
    args = ap.parse_args()
    os.makedirs(OUT_DIR, exist_ok=True)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "sweep":
        return {"ragged": run_ragged, "serving": run_serving, "precision": run_precision,
                "c1": run_c1, "decode": run_decode, "ga": run_ga}[args.workload](args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
