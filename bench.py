#!/usr/bin/env python3
"""Benchmark of the particle-learning cycle (arXiv 1212.1639) on GB300.

Workload (one "step" = one full cycle: weights, CDF, resampling, propagation):
the local-level model of the paper's Section 4 at scale -- one filter, N = 2^20
particles, FP32 state, systematic resampling, observations from a seeded
series of T = 1000 (x_0 = 0, sigma^2 = 1, tau^2 = 0.1), IG(3, 2) priors.

value  : particle-steps/s over the K timed cycles, device time from CUDA events
         on the filter's stream, inputs resident in HBM; the 90 MB working set
         fits in L2, so L2 is flushed (256 MB write) before every timed cycle,
         outside the events.
cycle_ms: median and p99 of the timed cycles, and the paper's statistic (the
         mean of the 5 closest to the median of the first 10).
e2e    : the same metric through the C ABI with host buffers: each step sends
         one observation from host memory and reads the posterior summaries
         back (pf_step_estimate), wall-clock timed.
roofline: the dominant kernel's algorithmic bytes per launch / its mean
         CUDA-event duration (pf_step_profiled), against the measured copy
         bandwidth in MEASURED_PEAKS.json.
Extra keys: the same cycle at N = 2^24 (the single-filter target size) and
with multinomial and stratified resampling; with the next cycle's weights
computed in the propagation (the series known ahead) at 2^20 and 2^24; with
adaptive resampling (ESS below n/2); the resampling kernel sweep (pf_resample,
N = 2^10..2^24, flat to degenerate weights); batched filters (4096 uneven filters, one
persistent launch per cycle, against per-filter launches); the served form
(10,000 streams under Poisson load, continuous batching, p50/p90/p99 latency;
and under an 8 GB budget where admission waits); FP32 against FP64 precision.

--impl reference times the CPU oracle (single-threaded) on a bounded sample of
the same workload.  Under torchrun every rank runs its own independent filter
(no collective on the data path; weak scaling).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle_steps_per_sec"
UNIT = "particle-steps/s"
N_DEFAULT = 1 << 20
T_SERIES = 1000
L2_FLUSH_BYTES = 256 << 20

# Algorithmic bytes per particle per launch, FP32 state: what each kernel must
# read and write for the method, the roofline numerators:
BYTES_PER_PARTICLE = {
    "weights": 12 + 4,            # read x, sigma2, tau2; write l
    "scan": 4 + 8,                # read l; write Q
    "spacing_scan": 8,            # write S
    "partition": 0,               # one merge-path split per 2048 merged elements
    "merge_systematic": 8 + 4,    # read Q; write ancestors
    "stratified": 8 + 4,          # read Q; write ancestors
    "merge_multinomial": 8 + 8 + 4,  # read Q and S; write ancestors
    "cutpoint_search": 8 + 4,     # read Q; write I
    "cutpoint_method": 4 + 8 + 4,  # read I, Q at the start; write ancestors
    "propagate": 4 + 28 + 28,     # read ancestor; gather 28 B record; write 28 B record
    "cdf_resample": 4 + 8 + 4,   # read l; write Q; write ancestors (l is read twice, the
                                  # second time mostly from L2)
    "propagate_weights_next": 4 + 28 + 28 + 4,  # propagate, and write the next cycle's l
    "estimate": 12,               # read x, sigma2, tau2 (posterior summaries)
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_DEFAULT)
    p.add_argument("--scheme", default="systematic")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the 2^24, multinomial, stratified, batched, precision and served lines")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--batched-only", action="store_true",
                   help="print only the batched-filters measurement (one JSON line)")
    p.add_argument("--served-only", action="store_true",
                   help="print only the served measurements (one JSON line)")
    p.add_argument("--served-seconds", type=float, default=60.0)
    p.add_argument("--precision-only", action="store_true",
                   help="print only the FP32-vs-FP64 precision report (one JSON line)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def phys_gpu(local=0):
    """nvidia-smi index of this process's GPU."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis and len(vis.split(",")) > local and vis.split(",")[local].isdigit():
        return int(vis.split(",")[local])
    return local


def pow2_label(n):
    return "2^%d" % (n.bit_length() - 1) if n & (n - 1) == 0 else str(n)


def kernels_hash():
    h = hashlib.sha256()
    for f in ("kernels.cuh", "device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1212_1639_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _recorded(kernel, what):
    """A per-particle figure of `kernel` from the committed ncu summary
    (profiles/traffic.txt); None if the kernels changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split(":", 1)
        rec[k.strip()] = v.strip()
    if rec.get("kernels_hash") != kernels_hash():
        return None
    key = "%s_%s_per_particle" % (kernel, what)
    return float(rec[key]) if key in rec else None


def recorded_traffic(kernel, n):
    """dram bytes per launch from the committed ncu summary, scaled to n
    particles; None if the kernels changed since the capture."""
    v = _recorded(kernel, "bytes")
    return None if v is None else v * n


def max_over_ranks(x, world, device="cuda"):
    """The maximum of a per-rank number over all ranks (the job's time is its
    slowest rank's); x itself on one rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def head_start(ms=2.0):
    """Keep the stream busy for about `ms` before the first timed cycle (a spin
    kernel, outside the events), so that the host has queued the timed cycles
    ahead of the device and no host enqueue gap lands inside an event pair."""
    import torch
    torch.cuda._sleep(int(ms * 1e-3 * 2.0e9))


def time_cycles(f, y_dev, start, K, stream, flush, per=None):
    """K timed cycles; L2 flushed before each, outside the events.  Returns the
    total ms; per (a list) receives each cycle's ms."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    head_start()
    for i in range(K):
        if flush is not None:
            flush.zero_()
        ev[i][0].record(stream)
        f.run(y_dev[start + i:start + i + 1])
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    if per is not None:
        per.extend(ms)
    return sum(ms)


def cycle_stats(per):
    """Median and p99 of per-cycle times, and the paper's statistic: the mean
    of the 5 runs closest to the median of the first 10 (Section 4)."""
    v = np.array(per)
    first = v[:10]
    med10 = np.median(first)
    closest = first[np.argsort(np.abs(first - med10))[:5]]
    return {"median_ms": round(float(np.median(v)), 5), "p99_ms": round(float(np.percentile(v, 99)), 5),
            "mean_of_5_closest_to_median_of_10_ms": round(float(closest.mean()), 5),
            "cycles": int(v.size)}


def bench_sweep(pf, synth, stream, reps=10):
    """The resampling kernel sweep: pf_resample on normalised FP32 weights with
    log-weights ~ N(0, s^2), N = 2^10 .. 2^24, resampled particles per second
    (CUDA events around each call on the stream; scratch from the stream's
    pool)."""
    import torch
    out = {}
    for scheme, s in (("systematic", 1.0), ("systematic", 0.1), ("systematic", 5.0),
                      ("multinomial", 1.0), ("stratified", 1.0)):
        row = {}
        for e in range(10, 25, 2):
            n = 1 << e
            w = torch.from_numpy(synth.sweep_weights(n, s, 7)).to("cuda")
            anc = torch.empty(n, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            for _ in range(2):
                pf.resample(w, 7, scheme=scheme, out=anc, stream=stream)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(reps)]
            for a, b in evs:
                a.record(stream)
                pf.resample(w, 7, scheme=scheme, out=anc, stream=stream)
                b.record(stream)
            torch.cuda.synchronize()
            ms = float(np.median([a.elapsed_time(b) for a, b in evs]))
            row["2^%d" % e] = {"ms": round(ms, 4), "particles_per_s": n / (ms / 1e3)}
        out["%s_s%g" % (scheme, s)] = row
    return out


def time_cycles_ahead(f, y, start, K, stream, flush):
    """K timed cycles whose propagation also computes the next cycle's
    weights (pf_step_ahead), each cycle after the first of the run finding its
    weights ready; L2 flushed before each, outside the events."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    f.step_ahead(float(y[start - 1]), float(y[start]))  # untimed: announces y[start]
    head_start()
    for i in range(K):
        if flush is not None:
            flush.zero_()
        ev[i][0].record(stream)
        f.step_ahead(float(y[start + i]), float(y[start + i + 1]))
        ev[i][1].record(stream)
    f.step(float(y[start + K]))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev)


def bench_fused(pf, n, stream, y, y_dev, flush, K, W, unfused_ms):
    """The same single-filter workload with the next cycle's weights computed
    in each propagation (the series is known ahead)."""
    import torch
    f = pf.Filter(n, seed=1639, scheme="systematic", precision="fp32", stream=stream)
    f.run(y_dev[:W])
    f.sync()
    ms = time_cycles_ahead(f, y, W + 1, K, stream, flush)
    f.step_profiled(float(y[W + K + 2]))
    acc = {}
    for i in range(5):
        if flush is not None:
            flush.zero_()
            torch.cuda.synchronize()
        t = W + K + 3 + i
        for k, v in f.step_profiled(float(y[t]), y_next=float(y[t + 1])).items():
            acc.setdefault(k, []).append(v)
    f.step(float(y[W + K + 8]))
    f.sync()
    f.close()
    prof = {k: sum(v) / len(v) for k, v in acc.items()}
    kern = {k: {"ms": round(v, 5), "gbs": round(BYTES_PER_PARTICLE[k] * n / (v / 1e3) / 1e9, 1)}
            for k, v in prof.items()}
    return {"value": n * K / (ms / 1e3), "unit": UNIT, "steps": K, "ms_per_step": ms / K,
            "speedup_vs_unfused": round(unfused_ms / (ms / K), 4),
            "l2": "flushed before every timed cycle" if flush is not None else
                  "inputs larger than L2 (no flush)",
            "kernels": kern}


def bench_adaptive(pf, n, stream, y, y_dev, flush, K, W, ess_frac=0.5):
    """The single-filter workload with adaptive resampling: resample only when
    the effective sample size drops below ess_frac * n."""
    import torch
    f = pf.Filter(n, seed=1639, scheme="systematic", precision="fp32", stream=stream,
                  ess_frac=ess_frac)
    f.run(y_dev[:W])
    f.sync()
    ms = time_cycles(f, y_dev, W, K, stream, flush)
    prof = kernel_profile(f, y, W + K, 5, flush)
    f.close()
    return {"value": n * K / (ms / 1e3), "unit": UNIT, "steps": K, "ms_per_step": ms / K,
            "ess_frac": ess_frac, "l2": "flushed before every timed cycle",
            "kernels": {k: round(v, 5) for k, v in prof.items()}}


def kernel_profile(f, y, start, P, flush):
    """Mean per-kernel durations (ms) over P profiled cycles."""
    import torch
    acc = {}
    for i in range(P):
        if flush is not None:
            flush.zero_()
            torch.cuda.synchronize()
        for k, v in f.step_profiled(float(y[start + i])).items():
            acc.setdefault(k, []).append(v)
    return {k: sum(v) / len(v) for k, v in acc.items()}


def run_config(pf, n, scheme, K, W, y, y_dev, rank, flush, stream):
    """The benchmarked filter after W warm-up cycles run exactly as the timed
    ones (each after an L2 flush; the first write of the flush buffer maps its
    pages, which must not happen inside the timed region)."""
    import torch
    f = pf.Filter(n, seed=1639 + rank, filter_id=rank, scheme=scheme, precision="fp32",
                  stream=stream)
    for i in range(W):
        if flush is not None:
            flush.zero_()
        f.run(y_dev[i:i + 1])
    f.sync()
    return f


def bench_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1212_1639_gb300 import pf, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)  # flushes and events go on the filters' stream
    n, K, W = args.n, args.steps, max(args.warmup, 3)
    total_steps = W + K + 64
    _, y = synth.local_level_series(1639, max(T_SERIES, total_steps), filter_id=rank)
    y_dev = torch.from_numpy(y).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    f = run_config(pf, n, args.scheme, K, W, y, y_dev, rank, flush, stream)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(phys_gpu(local))
    clk.start()
    time.sleep(0.5)  # the sampler's start-up (NVML initialisation) stays outside the timed region
    t_wall0 = time.perf_counter()
    per_cycle = []
    ms = time_cycles(f, y_dev, W, K, stream, flush, per=per_cycle)
    t_wall1 = time.perf_counter()
    clocks = clk.stop()
    if world > 1:
        ms = max_over_ranks(ms, world)
        dist.barrier()
    value = world * n * K / (ms / 1e3)

    # per-kernel durations (live, CUDA events on the filter's stream)
    prof = kernel_profile(f, y, W + K, 10, flush)
    kernels = {}
    hbm, hbm_kind = peaks()
    for kname, kms in prof.items():
        key = kname
        if kname == "merge":
            key = "merge_multinomial" if "multinomial" in args.scheme else "merge_systematic"
        byts = BYTES_PER_PARTICLE[key] * n
        kernels[kname] = {"ms": round(kms, 5), "bytes": byts,
                          "gbs": round(byts / (kms / 1e3) / 1e9, 1)}
    dom = max(prof, key=prof.get)
    dkey = "merge_multinomial" if dom == "merge" and "multinomial" in args.scheme else (
        "merge_systematic" if dom == "merge" else dom)
    achieved = kernels[dom]["gbs"]
    traffic = recorded_traffic(dkey, n)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm,
                "peak_kind": hbm_kind, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": traffic, "algorithmic_bytes": kernels[dom]["bytes"]}
    # the same kernel against instruction issue, its actual bound: thread
    # instructions per particle from the committed ncu capture, against one
    # warp instruction per scheduler per cycle (4 per SM) at the maximum SM
    # clock seen during the timed region
    inst = _recorded(dkey, "inst")
    if inst is not None and clocks.get("sm_max_mhz"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        peak_i = sms * 4 * 32 * clocks["sm_max_mhz"] * 1e6 / 1e12
        ach_i = inst * n / (prof[dom] / 1e3) / 1e12
        roofline["issue"] = {"inst_per_particle": inst, "achieved": round(ach_i, 2),
                             "peak": round(peak_i, 2), "unit": "T thread-instructions/s",
                             "frac": round(ach_i / peak_i, 4)}
    cycle_bytes = sum(v["bytes"] for v in kernels.values())
    cycle_ms = sum(prof.values())
    # the posterior summaries (pf_estimate: the reduction kernel and the
    # 104-byte copy), on the same stream after an L2 flush
    est_ms = []
    for i in range(5):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        f.estimate()
        e1.record(stream)
        torch.cuda.synchronize()
        est_ms.append(e0.elapsed_time(e1))
    est_mean = float(np.mean(est_ms[1:]))
    est_bytes = BYTES_PER_PARTICLE["estimate"] * n
    estimate = {"ms": round(est_mean, 5), "bytes": est_bytes,
                "gbs": round(est_bytes / (est_mean / 1e3) / 1e9, 1),
                "frac_of_peak": round(est_bytes / (est_mean / 1e3) / 1e9 / hbm, 4),
                "note": "pf_estimate: summary kernel plus the 104-byte copy; reads x, sigma^2, tau^2"}

    # end to end through the C ABI with host buffers
    fe = pf.Filter(n, seed=7 + rank, filter_id=rank, scheme=args.scheme, precision="fp32",
                   stream=stream)
    fe.run(y[:W])
    fe.sync()
    Ke = min(K, 100)
    e2e_s = 0.0
    for i in range(Ke):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        est = fe.step_estimate(float(y[W + i]))
        e2e_s += time.perf_counter() - t0
    assert est["t"] == W + Ke
    e2e_s = max_over_ranks(e2e_s, world)
    e2e = {"value": world * n * Ke / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8,
           "d2h_bytes_per_step": 104, "steps": Ke,
           "note": "pf_step_estimate per step: y from the host, the cycle, the summary reduction and "
                   "the 104-byte summary D2H in one graph, synchronised; L2 flushed before each step "
                   "outside the timer"}
    fe.close()

    extra = {}
    if not args.no_extra and rank == 0:
        # single-filter target size: 2^24 particles, working set 1.6 GB > L2
        n24 = 1 << 24
        f24 = pf.Filter(n24, seed=24, scheme=args.scheme, precision="fp32", stream=stream)
        # the first cycles after the prior draw are atypical (more heavy
        # particles in the resampling); they are timed apart, and the target
        # is measured on cycles 50.. of the series, a running filter's regime
        W24, K24 = 50, min(K, 50)
        first24 = []
        time_cycles(f24, y_dev, 0, 10, stream, None, per=first24)
        f24.run(y_dev[10:W24])
        f24.sync()
        ms24 = time_cycles(f24, y_dev, W24, K24, stream, None)
        prof24 = kernel_profile(f24, y, W24 + K24, 5, None)
        b24 = {k: BYTES_PER_PARTICLE["merge_systematic" if k == "merge" else k] * n24 for k in prof24}
        b24 = {k: max(v, 1) for k, v in b24.items()}
        extra["n_2p24"] = {
            "value": n24 * K24 / (ms24 / 1e3), "unit": UNIT, "steps": K24,
            "ms_per_step": ms24 / K24, "l2": "inputs larger than L2 (no flush)",
            "cycles_timed": "t = %d .. %d of the series" % (W24, W24 + K24 - 1),
            "first_10_cycles_ms": round(sum(first24) / len(first24), 5),
            "cycle_hbm_frac": round(sum(b24.values()) / (ms24 / K24 / 1e3) / 1e9 / hbm, 4),
            "kernels": {k: {"ms": round(v, 5), "gbs": round(b24[k] / (v / 1e3) / 1e9, 1)}
                        for k, v in prof24.items()}}
        f24.close()
        # multinomial resampling at the same size (116 B/particle with the
        # spacing prefix and its second CDF read), beside the systematic cycle
        fm24 = pf.Filter(n24, seed=25, scheme="multinomial", precision="fp32", stream=stream)
        fm24.run(y_dev[:W24])
        fm24.sync()
        msm24 = time_cycles(fm24, y_dev, W24, K24, stream, None)
        profm24 = kernel_profile(fm24, y, W24 + K24, 3, None)
        fm24.close()
        bm24 = sum(BYTES_PER_PARTICLE["merge_multinomial" if k == "merge" else k] * n24
                   for k in profm24)
        extra["n_2p24_multinomial"] = {
            "value": n24 * K24 / (msm24 / 1e3), "unit": UNIT, "steps": K24,
            "ms_per_step": msm24 / K24, "l2": "inputs larger than L2 (no flush)",
            "cycle_hbm_frac": round(bm24 / (msm24 / K24 / 1e3) / 1e9 / hbm, 4),
            "kernels": {k: round(v, 5) for k, v in profm24.items()}}
        # the series is known ahead: every propagation also computes the next
        # cycle's weights
        extra["fused_next_weights"] = bench_fused(pf, n, stream, y, y_dev, flush, min(K, 100), W,
                                                  ms / K)
        extra["n_2p24_fused_next_weights"] = bench_fused(pf, n24, stream, y, y_dev, None, K24, W24,
                                                         ms24 / K24)
        extra["adaptive_ess"] = bench_adaptive(pf, n, stream, y, y_dev, flush, min(K, 100), W)
        extra["resample_sweep"] = bench_sweep(pf, synth, stream)
        # the same workload with binary64 state (the paper's GPU(dp) column);
        # binary64 runs at a small fraction of the binary32 rate on GB300
        fd = pf.Filter(n, seed=3, scheme=args.scheme, precision="fp64", stream=stream)
        fd.run(y_dev[:W])
        fd.sync()
        Kd = min(K, 20)
        msd = time_cycles(fd, y_dev, W, Kd, stream, flush)
        profd = kernel_profile(fd, y, W + Kd, 3, flush)
        fd.close()
        extra["fp64"] = {"value": n * Kd / (msd / 1e3), "unit": UNIT, "steps": Kd,
                         "ms_per_step": msd / Kd, "kernels": {k: round(v, 5) for k, v in profd.items()}}
        for other in ("multinomial", "stratified"):  # the other resampling schemes
            if other == args.scheme:
                continue
            fm = pf.Filter(n, seed=3, scheme=other, precision="fp32", stream=stream)
            fm.run(y_dev[:W])
            fm.sync()
            Km = min(K, 100)
            msm = time_cycles(fm, y_dev, W, Km, stream, flush)
            profm = kernel_profile(fm, y, W + Km, 5, flush)
            extra[other] = {
                "value": n * Km / (msm / 1e3), "unit": UNIT, "steps": Km, "ms_per_step": msm / Km,
                "kernels": {k: round(v, 5) for k, v in profm.items()}}
            fm.close()
        extra["plain_config"] = bench_plain_config(pf, synth, stream)
        extra["batched"] = bench_batched(pf, synth, stream)
        extra["precision"] = bench_precision(pf, synth, stream)
        extra["served"] = bench_served(pf, synth, stream, duration=args.served_seconds)
        extra["served_admission"] = bench_served(pf, synth, stream, duration=20.0, budget_gb=8.0,
                                                 session_s=10.0)
        cap = bench_served_capacity(pf, synth, stream)
        per = bench_served_per_stream(pf, synth, stream)
        cap["per_stream_launches"] = per
        if cap["capacity_obs_per_s"]:
            cap["speedup_vs_per_stream_launches"] = round(cap["capacity_obs_per_s"] / per["obs_per_s"], 1)
        extra["served"]["capacity"] = cap
    f.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(n, args.scheme, y)

    launches_per_cycle = len(prof)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "local-level particle learning, one filter per GPU, "
                               "N=%s, FP32 state, %s resampling, T=1000 seeded series"
                               % (pow2_label(args.n), args.scheme),
                   "n_particles": n, "scheme": args.scheme, "precision": "fp32",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed (256 MB write) before every timed cycle, outside the events"},
        "roofline": roofline,
        "cycle": {"bytes": cycle_bytes, "ms_sum_of_kernels": round(cycle_ms, 5),
                  "hbm_frac_of_graph_time": round(cycle_bytes / (ms / K / 1e3) / 1e9 / hbm, 4),
                  "kernels": kernels},
        "e2e": e2e,
        "estimate": estimate,
        "cycle_ms": cycle_stats(per_cycle),
        "gpu_launches": launches_per_cycle * K,
        "clocks": clocks,
        "wall_s_timed": round(t_wall1 - t_wall0, 3),
    }
    line.update(extra)
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def bench_batched(pf, synth, stream, K=20, W=3, Kp=3, n_filters=4096, seed=4096):
    """Many uneven filters: one persistent launch per cycle (pf_batch_step)
    against per-filter launches of the plain cycle (pf_step on each filter).
    4096 filters, N log-uniform in [256, 65536], each with its own series
    simulated from true variances drawn from the IG(3, 2) prior; FP32,
    systematic.  Both forms give bit-identical results per filter."""
    import torch
    ns, s2, t2 = synth.batch_specs(n_filters, seed)
    T = W + max(K, Kp) + 1
    ys = np.stack([synth.local_level_series(seed + i, T, sigma2=s2[i], tau2=t2[i], filter_id=i)[1]
                   for i in range(n_filters)], axis=1)  # [T, filters]
    specs = [dict(n=int(ns[i]), seed=seed + i, filter_id=i) for i in range(n_filters)]
    total = int(ns.sum())
    b = pf.Batch(specs, scheme="systematic", precision="fp32", stream=stream)
    shapes, chosen = b.tune(ys[0])  # trial cycles: launch shape only, no result changes
    for t in range(W):
        b.step(ys[t])
    b.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for t in range(W, W + K):
        b.step(ys[t])
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms_b = ev[0].elapsed_time(ev[1]) / K
    info = b.info()
    b.close()
    torch.cuda.empty_cache()
    # per-filter launches of the plain cycle on the same stream
    fs = [pf.Filter(sp["n"], seed=sp["seed"], filter_id=sp["filter_id"], scheme="systematic",
                    precision="fp32", stream=stream) for sp in specs]
    for t in range(W):
        for i, f in enumerate(fs):
            f.step(ys[t, i])
    torch.cuda.synchronize()
    ev[0].record(stream)
    t0 = time.perf_counter()
    for t in range(W, W + Kp):
        for i, f in enumerate(fs):
            f.step(ys[t, i])
    ev[1].record(stream)
    torch.cuda.synchronize()
    wall_p = (time.perf_counter() - t0) / Kp
    ms_p = ev[0].elapsed_time(ev[1]) / Kp
    for f in fs:
        f.close()
    torch.cuda.empty_cache()
    hbm, _ = peaks()
    byts = total * (BYTES_PER_PARTICLE["weights"] + BYTES_PER_PARTICLE["scan"] +
                    BYTES_PER_PARTICLE["merge_systematic"] + BYTES_PER_PARTICLE["propagate"])
    return {
        "workload": "%d local-level filters, N log-uniform in [256, 65536] (sum %d), own series "
                    "from prior-drawn variances, FP32, systematic" % (n_filters, total),
        "value": total / (ms_b / 1e3), "unit": UNIT, "steps": K, "ms_per_step": ms_b,
        "gpu_launches_per_step": 1,
        "launch": {"grid": info["grid"], "block": info["block"], "cluster": info["cluster"],
                   "big_min": info["big_min"]},
        "autotune": {"chosen": chosen,
                     "shapes": [dict(sh, ms=round(sh["ms"], 4)) for sh in shapes]},
        "hbm_frac": round(byts / (ms_b / 1e3) / 1e9 / hbm, 4),
        "per_filter_launches": {"value": total / (ms_p / 1e3), "unit": UNIT, "steps": Kp,
                                "ms_per_step": ms_p, "host_wall_ms_per_step": wall_p * 1e3,
                                "gpu_launches_per_step": 5 * n_filters,
                                "note": "pf_step on each filter in turn, one stream"},
        "speedup_vs_per_filter": round(ms_p / ms_b, 2),
        "accuracy": "bit-identical per filter (tests/test_gpu_batch.py)",
        "cpu_baseline": oracle_batch_baseline(specs, ys),
    }


def bench_plain_config(pf, synth, stream, runs=10, T=100, n=1024):
    """The paper's plain configuration (its Section 4 run): one filter, N = 1024,
    T = 100, FP64 state, multinomial resampling.  Ten runs on the same series;
    each run creates the filter (the initialisation kernel) and runs the 100
    cycles.  Reported as the paper reports its runs: ms per 100-step run (the
    mean of the 5 runs closest to the median of the 10) and particle-steps/s,
    with the per-cycle device time beside it."""
    import torch
    _, y = synth.local_level_series(1212, T)
    y_dev = torch.from_numpy(y).cuda()
    walls, cyc = [], []
    for r in range(runs + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = pf.Filter(n, seed=1212, scheme="multinomial", precision="fp64", stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f.run(y_dev)
        e1.record(stream)
        f.sync()
        wall = time.perf_counter() - t0
        f.close()
        if r:  # the first run loads the kernels
            walls.append(wall * 1e3)
            cyc.append(e0.elapsed_time(e1) / T)
    w = np.array(walls)
    med = np.median(w)
    m5 = float(w[np.argsort(np.abs(w - med))[:5]].mean())
    return {"workload": "one filter, N=1024, T=100, FP64 state, multinomial resampling, "
                        "IG(3,2) priors, seeded series (the paper's plain configuration)",
            "value": n * T / (m5 / 1e3), "unit": UNIT, "ms_per_run": round(m5, 4),
            "run_statistic": "mean of the 5 runs closest to the median of 10 (wall clock, "
                             "filter creation and 100 cycles, synchronised)",
            "cycle_us_median": round(float(np.median(cyc)) * 1e3, 2),
            "cycle_device_particle_steps_per_s": n / (float(np.median(cyc)) / 1e3)}


def oracle_batch_baseline(specs, ys, cycles=3, max_filters=512):
    """The oracle on a sample of the batched workload (the first max_filters
    filters of the same batch, `cycles` cycles each), one host core and all
    host cores (one filter per thread; the oracle's calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle as orc
    sub = specs[:max_filters]
    total = sum(sp["n"] for sp in sub)
    out = {"sample": "%d filters (sum N = %d), %d cycles each" % (len(sub), total, cycles),
           "kind": "oracle", "unit": UNIT, "host": host_cpu()}
    ncpu = out["host"]["nproc"] or 1
    for cores in sorted({1, ncpu}):
        filters = [orc.Filter(orc.make_config(sp["n"], seed=sp["seed"], filter_id=sp["filter_id"],
                                              scheme=orc.SYSTEMATIC, precision=orc.FP32))
                   for sp in sub]

        def run(i):
            for t in range(cycles):
                filters[i].step(float(ys[t, i]))

        t0 = time.perf_counter()
        with ThreadPoolExecutor(cores) as ex:
            list(ex.map(run, range(len(sub))))
        dt = time.perf_counter() - t0
        for fo in filters:
            fo.close()
        out["cores_%d" % cores] = {"value": total * cycles / dt, "cores": cores}
    return out


def served_events(pf, synth, n_streams, duration, rate, seed, session_s=None):
    """Poisson observation events for n_streams streams (N log-uniform in
    [512, 131072], own series from prior-drawn variances).  Without
    session_s every stream is open for the whole run; with it, stream i is
    open for session_s seconds starting at a uniform time."""
    ns, s2, t2 = synth.batch_specs(n_streams, seed, 512, 131072)
    rng = np.random.default_rng([seed, 0x5E55])
    if session_s is None:
        start = np.zeros(n_streams)
        life = np.full(n_streams, duration)
    else:
        start = rng.random(n_streams) * (duration - session_s)
        life = np.full(n_streams, session_s)
    ts, ids, ys = [], [], []
    for i in range(n_streams):
        k = rng.poisson(rate * life[i])
        a = np.sort(rng.random(k)) * life[i] + start[i]
        ys.append(synth.local_level_series(seed + i, k, sigma2=s2[i], tau2=t2[i], filter_id=i)[1])
        ts.append(a)
        ids.append(np.full(k, i, np.uint64))
    t = np.concatenate([start] + ts + [start + life + 1e-3])
    kind = np.concatenate([np.full(n_streams, pf.EVENT_OPEN, np.uint8)] +
                          [np.zeros(len(a), np.uint8) for a in ts] +
                          [np.full(n_streams, pf.EVENT_CLOSE, np.uint8)])
    sid = np.concatenate([np.arange(n_streams, dtype=np.uint64)] + ids +
                         [np.arange(n_streams, dtype=np.uint64)])
    y = np.concatenate([np.zeros(n_streams)] + ys + [np.zeros(n_streams)])
    pri = np.where(kind == pf.EVENT_OPEN, 0, np.where(kind == pf.EVENT_CLOSE, 2, 1))
    order = np.lexsort((pri, t))
    cfgs = [dict(n=int(ns[i]), seed=seed + i, filter_id=i) for i in range(n_streams)]
    return t[order], kind[order], sid[order], y[order], cfgs, int(ns.sum())


def bench_served(pf, synth, stream, duration=60.0, budget_gb=120.0, n_streams=10000,
                 rate=20.0, seed=10000, session_s=None, cluster=8, big_min=16384, warmup_s=5.0):
    """Continuous-batching server under Poisson load: 10,000 streams at 20
    observations/s each (200k/s aggregate), device-resident state admitted
    under an HBM budget; throughput and latency percentiles."""
    import torch
    t, kind, sid, y, cfgs, total = served_events(pf, synth, n_streams, duration, rate, seed,
                                                 session_s)
    srv = pf.Server(max_streams=n_streams, hbm_budget_bytes=int(budget_gb * 1e9),
                    scheme="systematic", precision="fp32", max_inflight=2, cluster=cluster,
                    big_min=big_min, warmup_s=warmup_s, stream=stream)
    clk = Clocks(phys_gpu())
    clk.start()
    t0 = time.perf_counter()
    srv.replay(t, kind, sid, y, cfgs)
    srv.drain(duration + 600)
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    st = srv.stats()
    srv.close()
    torch.cuda.empty_cache()
    return {
        "workload": "%d streams, N log-uniform in [512, 131072] (sum %d), Poisson %.0f obs/s "
                    "per stream (%.0f/s aggregate) for %.0f s%s, FP32, systematic, budget %.0f GB"
                    % (n_streams, total, rate, rate * n_streams, duration,
                       "" if session_s is None else ", sessions of %.0f s" % session_s, budget_gb),
        "value": st["particle_steps_per_s"], "unit": UNIT,
        "obs_per_s": st["obs_per_s"], "observations": st["completed"],
        "latency_us": {"p50": round(st["p50_us"], 1), "p90": round(st["p90_us"], 1),
                       "p99": round(st["p99_us"], 1), "max": round(st["max_us"], 1),
                       "mean": round(st["mean_us"], 1)},
        "latency_us_after_warmup": {"warmup_s": warmup_s, "observations": st["steady_count"],
                                    "p50": round(st["steady_p50_us"], 1),
                                    "p90": round(st["steady_p90_us"], 1),
                                    "p99": round(st["steady_p99_us"], 1)},
        "cycles": st["cycles"], "mean_streams_per_cycle": round(st["mean_cycle_streams"], 1),
        "max_streams_per_cycle": st["max_cycle_streams"],
        "gpu_launches": 2 * st["cycles"],
        "launch": {"block": st["block"], "grid": st["grid"], "cluster": st["cluster"],
                   "big_min": big_min if st["cluster"] > 1 else None},
        "admission": {"admitted": st["admitted"], "admitted_after_wait": st["admitted_after_wait"],
                      "mean_wait_us": round(st["mean_admission_wait_us"], 1),
                      "pool_particles": st["pool_particles"]},
        "replay_max_lag_us": round(st["replay_max_lag_us"], 1), "wall_s": round(wall, 2),
        "clocks": clocks,
        "note": "latency = submit -> the stream's summaries on the host; each result equals "
                "the stream alone (tests/test_gpu_serve.py)",
    }


def bench_served_capacity(pf, synth, stream, rates=(20.0, 50.0, 80.0, 120.0), duration=4.0,
                          warmup_s=1.0, p99_bound_ms=10.0, n_streams=10000, seed=10000):
    """Capacity of the served form: the same 10,000 streams under Poisson
    loads of increasing rate (observations/s per stream) for `duration` s
    each; the capacity is the highest offered rate whose observations are all
    served at the offered rate with p99 latency (after the warm-up) within
    the bound."""
    import torch
    rows = []
    for r in rates:
        t, kind, sid, y, cfgs, total = served_events(pf, synth, n_streams, duration, r, seed)
        srv = pf.Server(max_streams=n_streams, hbm_budget_bytes=int(120e9), scheme="systematic",
                        precision="fp32", max_inflight=2, cluster=8, big_min=16384,
                        warmup_s=warmup_s, stream=stream)
        srv.replay(t, kind, sid, y, cfgs)
        srv.drain(duration + 600)
        st = srv.stats()
        srv.close()
        torch.cuda.empty_cache()
        offered = r * n_streams
        rows.append({"offered_obs_per_s": offered, "obs_per_s": round(st["obs_per_s"], 1),
                     "particle_steps_per_s": st["particle_steps_per_s"],
                     "p50_us": round(st["steady_p50_us"], 1), "p99_us": round(st["steady_p99_us"], 1),
                     "mean_streams_per_cycle": round(st["mean_cycle_streams"], 1)})
    ok = [row for row in rows if row["p99_us"] <= p99_bound_ms * 1e3
          and row["obs_per_s"] >= 0.97 * row["offered_obs_per_s"]]
    best = max(ok, key=lambda row: row["offered_obs_per_s"]) if ok else None
    return {"sweep": rows, "p99_bound_ms": p99_bound_ms, "duration_s": duration,
            "capacity_obs_per_s": best["obs_per_s"] if best else None,
            "capacity_particle_steps_per_s": best["particle_steps_per_s"] if best else None,
            "note": "highest offered rate served in full with p99 (after %.0f s) within %.0f ms; "
                    "above it the queue grows" % (warmup_s, p99_bound_ms)}


def bench_served_per_stream(pf, synth, stream, n_streams=256, rounds=3, seed=10000):
    """The served streams processed without the server: each stream a
    standalone filter, each round one observation per stream -- pf_step on
    every stream (plain-kernel launches, asynchronous), then pf_estimate on
    every stream for its result.  The same results as served (bit for bit,
    tests/test_gpu_serve.py); observations/s for comparison with the served
    capacity."""
    import torch
    ns, s2, t2 = synth.batch_specs(10000, seed, 512, 131072)
    ids = list(range(n_streams))
    ys = [synth.local_level_series(seed + i, rounds + 2, sigma2=s2[i], tau2=t2[i], filter_id=i)[1]
          for i in ids]
    fs = [pf.Filter(int(ns[i]), seed=seed + i, filter_id=i, scheme="systematic", precision="fp32",
                    stream=stream) for i in ids]
    for k, f in enumerate(fs):  # one untimed round: graphs captured
        f.step(ys[k][0])
        f.estimate()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in range(1, rounds + 1):
        for k, f in enumerate(fs):
            f.step(ys[k][r])
        for f in fs:
            f.estimate()
    dt = time.perf_counter() - t0
    for f in fs:
        f.close()
    torch.cuda.empty_cache()
    obs = n_streams * rounds
    total = int(sum(int(ns[i]) for i in ids))
    return {"streams": n_streams, "sum_n": total, "rounds": rounds,
            "obs_per_s": obs / dt, "particle_steps_per_s": total * rounds / dt,
            "gpu_launches_per_obs": 4,
            "note": "pf_step on each stream (asynchronous), then pf_estimate on each (its result); "
                    "the first %d streams of the served workload" % n_streams}


def bench_precision(pf, synth, stream, reps=8):
    """FP32 state against FP64 state on the same draws, per posterior summary
    and step, in units of the Monte Carlo sd of the estimate (the spread of
    FP64 filters over `reps` independent seeds).  FP64 filters equal the FP64
    oracle within 1e-12 at every step (tests/test_gpu_precision.py), so these
    are the FP32 errors against the FP64 oracle."""
    import torch
    keys = ("x_mean", "sigma2_mean", "tau2_mean", "log_marglik")
    out = {}
    for name, n, T, scheme, seed in (("N=1024, T=100, multinomial", 1024, 100, "multinomial", 1212),
                                     ("N=2^20, T=100, systematic", 1 << 20, 100, "systematic", 1639)):
        _, y = synth.local_level_series(seed, T)

        def path(sd, prec, anc_ref=None):
            f = pf.Filter(n, seed=sd, scheme=scheme, precision=prec, stream=stream)
            est, ancs = [], []
            for t in range(T):
                f.step(y[t])
                est.append([f.estimate()[k] for k in keys])
                if anc_ref is not None:
                    ancs.append(f.ancestors().cpu())
            f.close()
            return np.array(est), ancs

        e64, a64 = path(seed, "fp64", True)
        e32, a32 = path(seed, "fp32", True)
        first = next((t for t in range(T) if not torch.equal(a32[t], a64[t])), None)
        rep = np.stack([path(seed + 1000 + r, "fp64")[0] for r in range(reps)])
        mc = rep.std(axis=0, ddof=1)
        z = np.abs(e32 - e64) / mc
        out[name] = {
            "max_abs_err_in_mc_sd": dict(zip(keys, np.round(z.max(axis=0), 3).tolist())),
            "mean_abs_err_in_mc_sd": dict(zip(keys, np.round(z.mean(axis=0), 3).tolist())),
            "final": {k: {"fp64": float(e64[-1, i]), "fp32": float(e32[-1, i]),
                          "mc_sd": float(mc[-1, i])} for i, k in enumerate(keys)},
            "first_step_fp32_ancestors_differ": first}
    out["note"] = ("FP32-state against FP64-state filters with the same seeds; errors in units of "
                   "the Monte Carlo sd measured over %d FP64 seeds; FP64 equals the FP64 oracle "
                   "within 1e-12 (tests/test_gpu_precision.py)" % reps)
    return out


def host_cpu():
    """The host CPU the oracle runs on: model name (lscpu, else /proc/cpuinfo)
    and the number of cores the process may use."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    ncpu = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"model": model, "nproc": ncpu, "machine": os.uname().machine}


def cpu_baseline(n, scheme, y, budget_s=15.0):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    workload: the same N and series, as many cycles as fit in ~budget_s."""
    from oracle import oracle as orc

    sch = {"systematic": orc.SYSTEMATIC, "multinomial": orc.MULTINOMIAL,
           "systematic_cutpoint": orc.SYSTEMATIC_CUTPOINT,
           "multinomial_cutpoint": orc.MULTINOMIAL_CUTPOINT}[scheme]
    o = orc.Filter(orc.make_config(n, seed=1639, scheme=sch, precision=orc.FP32))
    steps, t0 = 0, time.perf_counter()
    while steps < 3 or (time.perf_counter() - t0 < budget_s and steps < 200):
        o.step(y[steps])
        steps += 1
    dt = time.perf_counter() - t0
    o.close()
    return {"value": n * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "N=%d particles, first %d cycles of the same series (FP32 state, %s)"
                      % (n, steps, scheme), "host": host_cpu()}


def bench_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_1212_1639_gb300 import synth

    n = args.n
    # each step is one cycle of the workload; the particle count is the full
    # 2^20 so each step costs ~0.3 s of CPU -- bound the run to a few minutes
    K = min(args.steps, 200)
    W = min(args.warmup, 3)
    _, y = synth.local_level_series(1639, max(T_SERIES, W + K + 1))
    sch = {"systematic": orc.SYSTEMATIC, "multinomial": orc.MULTINOMIAL}.get(args.scheme, orc.SYSTEMATIC)
    o = orc.Filter(orc.make_config(n, seed=1639, scheme=sch, precision=orc.FP32))
    for i in range(W):
        o.step(y[i])
    t0 = time.perf_counter()
    deadline = t0 + 240.0
    done = 0
    for i in range(K):
        o.step(y[W + i])
        done += 1
        if time.perf_counter() > deadline:
            break
    dt = time.perf_counter() - t0
    value = n * done / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": done, "warmup": W, "ms_per_step": dt * 1e3 / done, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "local-level particle learning, one filter per GPU, "
                               "N=%s, FP32 state, %s resampling, T=1000 seeded series"
                               % (pow2_label(n), args.scheme),
                   "n_particles": n, "scheme": args.scheme, "precision": "fp32"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "N=%d, %d cycles (of %d requested) on one host core"
                                   % (n, done, K)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        bench_reference(args)
    elif args.batched_only:
        import torch

        from paper_1212_1639_gb300 import pf, synth
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        print(json.dumps(bench_batched(pf, synth, stream, K=args.steps, W=max(args.warmup, 3))))
    elif args.precision_only:
        import torch

        from paper_1212_1639_gb300 import pf, synth
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        print(json.dumps(bench_precision(pf, synth, stream)))
    elif args.served_only:
        import torch

        from paper_1212_1639_gb300 import pf, synth
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        print(json.dumps({
            "served": bench_served(pf, synth, stream, duration=args.served_seconds),
            "served_no_clusters": bench_served(pf, synth, stream, duration=args.served_seconds,
                                               cluster=1),
            "served_admission": bench_served(pf, synth, stream, duration=20.0, budget_gb=8.0,
                                             session_s=10.0),
            "capacity": bench_served_capacity(pf, synth, stream),
            "per_stream_launches": bench_served_per_stream(pf, synth, stream)}))
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
