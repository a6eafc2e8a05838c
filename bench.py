"""Benchmark of the batched AM loop (one JSON line on stdout).

One step = one solve of the paper-shaped workload: 1000 trajectories, 100
steps over 10 s, 3 robot circles, 10 moving ellipses, 100 AM iterations
(position QP, heading QP, closed-form alpha/d steps, residual, cost and
multiplier updates), then the best-trajectory selection.  Inputs are the
seeded synthetic workload; they are resident on the GPU before the timed
region, and a 512 MiB buffer is rewritten between timed steps to flush L2.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank solves its own 1000-trajectory batch (weak scaling,
no data-path collective); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "trajectory-AM-iterations/sec at batch 1000; p50/p99 re-plan latency vs plain GPU"
UNIT = "trajectory-iterations/s"
WORKLOAD = "paper"
B, ITERS = 1000, 100


def algorithmic_flops(q: int, m: int, n: int) -> float:
    """FP32 flops of one AM iteration for one trajectory (FMA = 2 flops),
    counted from the formulas of the trig-free form, independent of how the
    kernel schedules them:
      obstacle pairs  17 per (circle, obstacle, step): scaled offset (2 FMA),
                      squared distance (2 FMA), rsqrt, max and subtract,
                      offset scaling (2), accumulation (2 FMA)
      circles         16 per (circle, step): circle centre (2 FMA), residual
                      rows (3 FMA... ) and their two weighted sums
      bounds          16 per step: two norms, rsqrt, clips, projected values
      trajectories    176 per step: 8 values x 11 coefficients (FMA)
      heading         66 per step + 2 x 121: W^T delta, P^T delta, psi = P xi2
      contraction     176 per step: R = F^T (g - F xi1), 88 dots per step
      position step   3960: 44 rows x 44 FMA, multiplier update 44 FMA
    """
    return 17.0 * m * n * q + 16.0 * m * q + (16 + 176 + 66 + 176) * q + 2 * 121 * 2 + 3960.0


def survey_flops(q: int, m: int, n: int) -> float:
    """The scope table's per-unit figure for one AM iteration of one
    trajectory (its bounding-roofline estimate): 28 flop per (circle,
    obstacle, step) element of the obstacle sweep, plus the contractions --
    F^T g (2 sides x 2 x 11 x 4 per step), the basis evaluation (8 x 2 x 11
    per step), the heading step (70 per step) and the KKT products (4000
    per trajectory).  130,200 at q = 100, m = 3, n = 10."""
    return 28.0 * m * n * q + (176 + 176 + 70) * q + 4000.0


def measured_traffic(profile: str = "am_warp_kernel_paper_b1000.md", source: str = "am_warp.cu"):
    """DRAM bytes per launch of a kernel from its committed ncu summary, if
    that summary was taken on the current kernel source (else None)."""
    import hashlib
    import re
    prof = os.path.join(ROOT, "profiles", profile)
    src = os.path.join(ROOT, "paper_2109_13030_b300", "csrc", source)
    try:
        text = open(prof).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    m = re.search(re.escape(source) + r": `([0-9a-f]{16})`", text)
    t = re.search(r"dram__bytes_read.sum / write.sum \| ([\d,]+) B / ([\d,]+) B", text)
    if not m or not t or m.group(1) != sha:
        return None
    return int(t.group(1).replace(",", "")) + int(t.group(2).replace(",", ""))


def large_profile():
    """Tensor-pipe share and DRAM bytes per launch of the large-batch kernel
    from its committed ncu summary, if taken on the current kernel source."""
    import hashlib
    import re
    prof = os.path.join(ROOT, "profiles", "am_large_kernel_paper_b18944.md")
    src = os.path.join(ROOT, "paper_2109_13030_b300", "csrc", "am_large.cu")
    try:
        text = open(prof).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    m = re.search(r"am_large.cu: `([0-9a-f]{16})`", text)
    t = re.search(r"sm__pipe_tensor_cycles_active \| ([\d.]+) %", text)
    d = re.search(r"dram__bytes_read.sum / write.sum \| ([\d,]+) B / ([\d,]+) B", text)
    if not m or m.group(1) != sha:
        return None
    out = {}
    if t:
        out["tensor_pipe_pct"] = float(t.group(1))
    if d:
        out["traffic"] = int(d.group(1).replace(",", "")) + int(d.group(2).replace(",", ""))
    return out or None


def sig(x, n: int = 4):
    """x rounded to n significant digits (None and non-numbers unchanged)."""
    if isinstance(x, bool) or not isinstance(x, (int, float)) or x == 0 or not np.isfinite(x):
        return x
    return float(f"{x:.{n}g}")


def compact(d):
    """Every float in a nested dict/list rounded to 4 significant digits."""
    if isinstance(d, dict):
        return {k: compact(v) for k, v in d.items()}
    if isinstance(d, list):
        return [compact(v) for v in d]
    return sig(d) if isinstance(d, float) else d


def summary_sections(extra: dict) -> dict:
    """Short forms of the single-GPU sections, so that the whole JSON line stays
    within a few kilobytes: throughput and times, p50/p99 per serving mode."""
    out = {}
    if "uneven" in extra:
        u = extra["uneven"]
        out["uneven"] = {"value": u["value"], "ms": u["ms_per_solve"], "precision": u.get("precision", "fp32"),
                         "threads": u["threads"], "launches": u["launches_per_solve"],
                         "per_problem_value": u["one_launch_per_problem"]["value"],
                         "per_problem_ms": u["one_launch_per_problem"]["ms_per_solve"]}
        if "bf16" in u:
            out["uneven"]["bf16_value"] = u["bf16"]["value"]
            out["uneven"]["bf16_ms"] = u["bf16"]["ms_per_solve"]
        if "auto" in u:
            out["uneven"]["auto_value"] = u["auto"]["value"]
            out["uneven"]["auto_ms"] = u["auto"]["ms_per_solve"]
            out["uneven"]["auto_slots_cap"] = u["auto"].get("warp_slots_cap")
            out["uneven"]["auto_frac"] = u["auto"].get("frac_of_fp32_peak")
            out["uneven"]["auto_frac_finer"] = u["auto"].get("frac_finer_count")
    if "precision" in extra:
        pr = extra["precision"]
        out["precision_b4096"] = {k: {"value": v["value"], **({"dev10": v["coef_dev_vs_fp32_after_10"]["max"]}
                                                              if "coef_dev_vs_fp32_after_10" in v else {})}
                                  for k, v in pr.items() if isinstance(v, dict)}
    if "large" in extra:
        lg = extra["large"]
        out["large_batch"] = {k: {"large": v["large"]["value"], "small_tile": v["small_tile"]["value"],
                                  "warp_pair": v["warp_pair"]["value"],
                                  "large_ms": v["large"]["kernel_ms"], "frac": v["large"]["frac_of_fp32_peak"]}
                              for k, v in lg.items() if k.startswith("B=")}
        if lg.get("profile"):
            out["large_batch"]["profile"] = lg["profile"]
    if "serving" in extra:
        sv = extra["serving"]
        pq = lambda r: [r["p50_ms"], r["p99_ms"]]
        out["serving_p50_p99_ms"] = {
            "400/s": {"batched": pq(sv["batched"]), "seq_fused": pq(sv["sequential_fused"]),
                      "batched_auto": pq(sv["batched_auto"]), "seq_auto": pq(sv["sequential_auto"]),
                      "seq_plain": pq(sv["sequential_plain_fp32_loop"])},
            # three runs each: [p50 per run], [p99 per run]
            "2500/s": {k: [[r["p50_ms"] for r in sv["high_load"][name]], [r["p99_ms"] for r in sv["high_load"][name]]]
                       for k, name in (("batched", "batched"), ("seq_fused", "sequential_fused"),
                                       ("batched_auto", "batched_auto"), ("seq_auto", "sequential_auto"))}}
        out["serving_mean_batch"] = {"400/s": sv["batched"]["mean_batch"],
                                     "2500/s": [r["mean_batch"] for r in sv["high_load"]["batched"]]}
        out["serving_submit_lag_max_ms"] = max(
            [sv[k]["submit_lag_max_ms"] for k in ("batched", "sequential_fused", "batched_auto", "sequential_auto")]
            + [r["submit_lag_max_ms"] for k, v in sv["high_load"].items() if isinstance(v, list) for r in v])
    return out


def peak_fp32_tflops(sms: int = 148, clock_mhz: float = 2032.0) -> float:
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sms * 128 * 2 * clock_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        time.sleep(0.25)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            # the reader thread ends at the pipe's end of file; join it and close
            # the pipe so that nothing of the sampler outlives the timed region
            self.thread.join(timeout=5)
            self.proc.stdout.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(pb, sample_B: int, iters: int, min_seconds: float = 10.0) -> dict:
    """The FP64 oracle (plain C, threads over trajectories, all host cores) on
    a bounded sample of the same workload: solves of the first sample_B
    trajectories, repeated until at least min_seconds of wall time."""
    from oracle import oracle as O
    sub = dict(pb)
    sub["init"] = pb["init"][:sample_B]
    sub["B"] = sample_B
    cores = os.cpu_count() or 1
    reps, dt = 0, 0.0
    while reps == 0 or dt < min_seconds:
        t0 = time.perf_counter()
        O.solve(sub, iters, nthreads=cores)
        dt += time.perf_counter() - t0
        reps += 1
    return {"value": reps * sample_B * iters / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} solve(s) of {sample_B} of the {pb['B']} trajectories x {iters} iterations, "
                      f"{dt:.1f} s wall"}


def bench_uneven(TJ, W, torch, dev, flush, steps: int, iters: int = 100) -> dict:
    """64 problems of mixed shape (B 128..2048, q in {50, 100, 150}, 2..32
    moving ellipses, 2..4 circles), 100 iterations each: one grouped launch
    (autotuned block size, replayed CUDA graph on a side stream) against one
    fused launch per problem on the same stream."""
    pbs = W.make_uneven(0, count=64)
    side = torch.cuda.Stream(dev)
    probs = [TJ.Problem(pb) for pb in pbs]
    inits = [torch.tensor(pb["init"], dtype=torch.float32, device=dev) for pb in pbs]

    def reset():
        for P, x in zip(probs, inits):
            P.init_state(x, stream=side)

    reset()
    G = TJ.Group(probs)
    threads, _ = G.autotune(iters, stream=side)
    for _ in range(2):
        reset()
        G.solve(iters, stream=side)
    torch.cuda.synchronize()
    launches0, items = G.stats()
    ms = []
    for i in range(steps):
        flush.fill_(float(i))
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        G.solve(iters, stream=side)
        e1.record(side)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    launches = (G.stats()[0] - launches0) / steps
    seq = []
    for i in range(steps):
        flush.fill_(float(i))
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        for P in probs:
            TJ.am_solve_batch(P.h, P.B, None, None, iters, side)
        e1.record(side)
        torch.cuda.synchronize()
        seq.append(e0.elapsed_time(e1))
    total = sum(pb["B"] for pb in pbs)
    flops = sum(algorithmic_flops(pb["q"], pb["m"], pb["n"]) * pb["B"] for pb in pbs) * iters
    flops_scope = sum(survey_flops(pb["q"], pb["m"], pb["n"]) * pb["B"] for pb in pbs) * iters
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    g_ms, s_ms = statistics.mean(ms), statistics.mean(seq)
    G.close()
    for P in probs:
        P.close()
    # the same mix with the contraction R in one BF16 tensor-core product
    # (the uneven-batching configuration's precision form)
    probs = [TJ.Problem(pb, precision=TJ.AM_BF16) for pb in pbs]
    reset()
    G = TJ.Group(probs)
    G.autotune(iters, stream=side)
    for _ in range(2):
        reset()
        G.solve(iters, stream=side)
    torch.cuda.synchronize()
    bms = []
    for i in range(steps):
        flush.fill_(float(i))
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        G.solve(iters, stream=side)
        e1.record(side)
        torch.cuda.synchronize()
        bms.append(e0.elapsed_time(e1))
    b_ms = statistics.mean(bms)
    G.close()
    for P in probs:
        P.close()
    # the same mix with AM_KERNEL_AUTO handles: every problem on the
    # warp-pair group kernels (two warps per trajectory for q <= 128, three
    # for q = 150), in one launch (FP32)
    probs = [TJ.Problem(pb, kernel=TJ.AM_KERNEL_AUTO) for pb in pbs]
    reset()
    G = TJ.Group(probs)
    G.autotune(iters, stream=side)   # here: the cap on the warp-pair kernels' slots per CTA
    a_slots = G.warp_slots()
    for _ in range(2):
        reset()
        G.solve(iters, stream=side)
    torch.cuda.synchronize()
    a_launch0, _ = G.stats()
    ams = []
    for i in range(steps):
        flush.fill_(float(i))
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        G.solve(iters, stream=side)
        e1.record(side)
        torch.cuda.synchronize()
        ams.append(e0.elapsed_time(e1))
    a_ms = statistics.mean(ams)
    a_launches = (G.stats()[0] - a_launch0) / steps
    G.close()
    for P in probs:
        P.close()
    return {"metric": "trajectory-AM-iterations/sec over 64 mixed problems", "value": total * iters / (g_ms / 1e3),
            "bf16": {"value": total * iters / (b_ms / 1e3), "unit": UNIT, "ms_per_solve": b_ms},
            "auto": {"value": total * iters / (a_ms / 1e3), "unit": UNIT, "ms_per_solve": a_ms,
                     "launches_per_solve": a_launches, "warp_slots_cap": a_slots,
                     "frac_of_fp32_peak": flops_scope / (a_ms / 1e3) / 1e12 / peak_fp32_tflops(sms),
                     "frac_finer_count": flops / (a_ms / 1e3) / 1e12 / peak_fp32_tflops(sms),
                     "problems_two_warps": sum(1 for pb in pbs if pb["q"] <= 128),
                     "problems_three_warps": sum(1 for pb in pbs if 128 < pb["q"] <= 192)},
            "unit": UNIT, "ms_per_solve": g_ms, "problems": len(pbs), "trajectories": total,
            "iterations": iters, "work_items": items, "threads": threads, "launches_per_solve": launches,
            "achieved_tflops": flops / (g_ms / 1e3) / 1e12,
            "one_launch_per_problem": {"value": total * iters / (s_ms / 1e3), "unit": UNIT,
                                       "ms_per_solve": s_ms, "launches_per_solve": len(pbs)},
            "workload": "make_uneven(seed 0, 64 problems): B uniform over 128..2048, q in {50,100,150}, "
                        "T=q/10 s, n 2..32 moving ellipses, m 2..4 circles over [-0.4, 0.4]"}


def bench_precision(TJ, W, torch, dev, flush, steps: int, iters: int = 100) -> dict:
    """The paper-shaped scene at B = 4096 in the four precision forms of the
    contraction R: FP32 (three TF32 products), one TF32 or BF16 product, and
    split BF16 (three BF16 products of K = 16).  Reports the fused kernel's time and
    each reduced form's coefficient deviation from the FP32 form after 10
    iterations (the error against the FP64 oracle is measured by the tests)."""
    pb = W.make_problem("precision", 0)
    Bp = pb["B"]
    init = torch.tensor(pb["init"], dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    out, ref = {}, None
    # the reduced forms act on the small-tile kernel's tensor-core product;
    # the warp-pair kernel (FP32 SIMT contractions) is timed beside them
    for prec, name, kern in ((TJ.AM_FP32, "fp32", TJ.AM_KERNEL_FUSED), (TJ.AM_TF32, "tf32", TJ.AM_KERNEL_FUSED),
                             (TJ.AM_BF16, "bf16", TJ.AM_KERNEL_FUSED),
                             (TJ.AM_SPLIT_BF16, "split_bf16", TJ.AM_KERNEL_FUSED),
                             (TJ.AM_FP32, "fp32_warp_pair", TJ.AM_KERNEL_WARP)):
        P = TJ.Problem(pb, precision=prec, kernel=kern)
        P.solve(init, 10, stream=stream)
        xi = P.state()[:, :55].astype(np.float64)
        ms = []
        for i in range(steps + 2):
            flush.fill_(float(i))
            TJ.am_init_state(P.h, Bp, init, None, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            TJ.am_solve_batch(P.h, Bp, None, None, iters, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        P.close()
        k_ms = statistics.mean(ms[2:])
        row = {"value": Bp * iters / (k_ms / 1e3), "unit": UNIT, "kernel_ms": k_ms}
        if ref is None:
            ref = xi
        else:
            dev_ = np.max(np.abs(xi - ref), axis=1) / np.maximum(np.max(np.abs(ref), axis=1), 1.0)
            row["coef_dev_vs_fp32_after_10"] = {"max": float(dev_.max()), "median": float(np.median(dev_))}
        out[name] = row
    out["workload"] = "paper-shaped scene at B = 4096, 100 iterations per timed solve"
    return out


def bench_large(TJ, W, torch, dev, flush, steps: int, iters: int = 100) -> dict:
    """The large-batch kernel (AM_KERNEL_LARGE: 128 trajectories per CTA, the
    contractions on tcgen05 tensor cores) on the paper-shaped scene at B =
    16384 and at one full wave (128 trajectories per SM), beside the
    small-tile and warp-pair fused kernels on the same batch.  Times are CUDA events around
    the solve on its stream, the initial state re-made and L2 flushed before
    each."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = peak_fp32_tflops(sms)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for Bl in (16384, 128 * sms):
        pb = W.make_problem("paper", 0, B=Bl)
        init = torch.tensor(pb["init"], dtype=torch.float32, device=dev)
        row = {}
        for kern, name in ((TJ.AM_KERNEL_LARGE, "large"), (TJ.AM_KERNEL_FUSED, "small_tile"),
                           (TJ.AM_KERNEL_WARP, "warp_pair")):
            P = TJ.Problem(pb, kernel=kern)
            ms = []
            for i in range(steps + 2):
                flush.fill_(float(i))
                P.init_state(init, stream=stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                TJ.am_solve_batch(P.h, Bl, None, None, iters, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            res_med = float(np.median(P.results()["res"]))
            P.close()
            k_ms = statistics.mean(ms[2:])
            row[name] = {"value": Bl * iters / (k_ms / 1e3), "kernel_ms": k_ms, "res_median": res_med}
        achieved = survey_flops(pb["q"], pb["m"], pb["n"]) * Bl * iters / (row["large"]["kernel_ms"] / 1e3) / 1e12
        fine = algorithmic_flops(pb["q"], pb["m"], pb["n"]) * Bl * iters / (row["large"]["kernel_ms"] / 1e3) / 1e12
        row["large"]["achieved_tflops"] = achieved
        row["large"]["frac_of_fp32_peak"] = achieved / peak
        row["large"]["frac_finer_count"] = fine / peak
        out[f"B={Bl}"] = row
    out["profile"] = large_profile()
    out["workload"] = "paper-shaped scene, 100 iterations per timed solve"
    return out


def serve_run(TJ, W, pbs, mode, kernel, seconds, warmup_s=1.0, rate=400.0, iters=30, seed=7):
    """One serving run: 64 resident scenes, Poisson arrivals at `rate`/s for
    warmup_s + seconds; each request picks a scene uniformly, moves its
    obstacles 0.1 s further along their (linear) tracks and starts the plan
    from the scene's last best plan at t = 0.1 s.  Latency is the server's
    submit-to-result time; requests arriving in the warm-up are not counted."""
    S = TJ.Server(8 << 30, iters, mode=mode)
    probs = []
    for pb in pbs:
        P = TJ.Problem(pb, kernel=kernel)
        S.add_scene(P, pb["init"].astype(np.float32))
        probs.append(P)
    S.start()
    rng = np.random.default_rng(seed)
    total = warmup_s + seconds
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(total * rate * 1.5) + 16))
    arrivals = arrivals[arrivals < total]
    picks = rng.integers(0, len(pbs), size=len(arrivals))
    vel = [((pb["xo"][:, -1] - pb["xo"][:, 0]) / pb["T"], (pb["yo"][:, -1] - pb["yo"][:, 0]) / pb["T"])
           for pb in pbs]
    clock = np.zeros(len(pbs))
    tickets = []
    # no collector pause inside the arrival loop: a pause would release the
    # requests it delayed as one burst
    gc_on = gc.isenabled()
    gc.disable()
    try:
        t0 = time.perf_counter()
        for a, k in zip(arrivals, picks):
            while True:
                dt = t0 + a - time.perf_counter()
                if dt <= 0:
                    break
                time.sleep(min(dt, 5e-4))
            clock[k] += 0.1
            pb = pbs[k]
            xo = (pb["xo"] + clock[k] * vel[k][0][:, None]).astype(np.float32)
            yo = (pb["yo"] + clock[k] * vel[k][1][:, None]).astype(np.float32)
            tickets.append((a, S.submit(int(k), advance=0.1, xo=xo, yo=yo)))
    finally:
        if gc_on:
            gc.enable()
    res = [(a, S.wait(t, timeout_s=300.0)) for a, t in tickets]
    stats = S.stats()
    S.close()
    for P in probs:
        P.close()
    bad = sum(1 for _, r in res if r["status"] != 0)
    lat = np.array([r["t_done"] - r["t_submit"] for a, r in res if a >= warmup_s]) * 1e3
    span = max(r["t_done"] for _, r in res) - min(r["t_submit"] for _, r in res)
    # how late the generator submitted each request against its schedule
    # (the server's clock and perf_counter are both the monotonic clock)
    lag = max(r["t_submit"] - (t0 + a) for a, r in res) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "requests_measured": int(len(lat)), "requests": len(res),
            "submit_lag_max_ms": float(lag),
            "failed": bad, "offered_per_s": rate, "served_per_s": len(res) / span,
            "rounds": stats["rounds"], "mean_batch": float(np.mean([r["batch"] for _, r in res])),
            "seconds": seconds, "warmup_s": warmup_s}


def bench_serving(TJ, W, seconds: float, plain_seconds: float) -> dict:
    pbs = W.make_uneven(0, count=64)
    out = {"metric": "re-plan latency (submit to result on the host)", "unit": "ms",
           "workload": "64 resident scenes of the mixed workload (B 128..2048, q in {50,100,150}, "
                       "n 2..32, m 2..4), Poisson arrivals at 400/s, 30 warm-started iterations per "
                       "request, obstacles +0.1 s and start state from the last best plan at +0.1 s, "
                       "8 GB budget",
           "iterations_per_request": 30}
    out["batched"] = serve_run(TJ, W, pbs, TJ.AM_SRV_BATCHED, TJ.AM_KERNEL_FUSED, seconds)
    out["sequential_fused"] = serve_run(TJ, W, pbs, TJ.AM_SRV_SEQUENTIAL, TJ.AM_KERNEL_FUSED, seconds)
    # scenes selecting AM_KERNEL_AUTO (warp-pair kernels where they take the scene)
    out["batched_auto"] = serve_run(TJ, W, pbs, TJ.AM_SRV_BATCHED, TJ.AM_KERNEL_AUTO, seconds)
    out["sequential_auto"] = serve_run(TJ, W, pbs, TJ.AM_SRV_SEQUENTIAL, TJ.AM_KERNEL_AUTO, seconds)
    out["sequential_plain_fp32_loop"] = serve_run(TJ, W, pbs, TJ.AM_SRV_SEQUENTIAL, TJ.AM_KERNEL_PLAIN,
                                                  plain_seconds)
    # a heavier load, where requests arrive while others are on the GPU and
    # rounds of continuous batching hold several of them
    # (three runs of each mode, different arrival seeds, so that the spread
    # of the tail shows)
    hi_rate = 2500.0
    out["high_load"] = {"offered_per_s": hi_rate, "runs": 3}
    for name, mode, kern in (("batched", TJ.AM_SRV_BATCHED, TJ.AM_KERNEL_FUSED),
                             ("sequential_fused", TJ.AM_SRV_SEQUENTIAL, TJ.AM_KERNEL_FUSED),
                             ("batched_auto", TJ.AM_SRV_BATCHED, TJ.AM_KERNEL_AUTO),
                             ("sequential_auto", TJ.AM_SRV_SEQUENTIAL, TJ.AM_KERNEL_AUTO)):
        out["high_load"][name] = [serve_run(TJ, W, pbs, mode, kern, plain_seconds, warmup_s=1.0, rate=hi_rate,
                                            seed=7 + rep) for rep in range(3)]
    return out


def bench_closed_loop(episodes: int, cem_episodes: int, seconds: float = 20.0, batches=(1, 200, 1000)) -> dict:
    """Closed-loop MPC on the crowd benchmarks of Sec. IV (Table III's
    metrics against batch size): `episodes` scenes per benchmark (static,
    same-direction, opposite flow), 20 s at 10 Hz, 10 iterations per re-plan,
    all episodes served together by one re-planning server."""
    from paper_2109_13030_b300 import mpc as M
    from paper_2109_13030_b300 import workload as W
    crowds = [W.make_crowd(k, s) for k in W.CROWD_KINDS for s in range(episodes)]
    cfg = M.MPCConfig(duration=seconds)
    out = {"workload": f"{len(crowds)} synthetic crowd episodes ({episodes} per benchmark: static, same-direction "
                       "flow <= 0.3 m/s, opposite flow <= 1.0 m/s; 30 people of radius 0.3 m in a 10 m band), "
                       f"robot of 3 circles tracking (t m/s, 0), {seconds:g} s at 10 Hz",
           "config": {"iters_per_replan": cfg.iters, "horizon_s": cfg.horizon, "q": cfg.q,
                      "planning_margin_m": cfg.margin,
                      "warm_start": "coefficients kept and re-timed, multipliers kept",
                      "fallback": "most clearance"},
           "by_batch": {}}
    for batch in batches:
        r = M.run(crowds, M.MPCConfig(batch=batch, duration=seconds))
        row = M.summarize(r["episodes"])
        row["by_benchmark_success"] = {k: M.summarize([e for e in r["episodes"] if e["kind"] == k])["success_rate"]
                                       for k in W.CROWD_KINDS}
        row["replan_ms"] = r["replan_ms"]
        row["control_steps"] = r["steps"]
        row["loop_wall_s"] = r["wall_s"]
        out["by_batch"][str(batch)] = row
    if cem_episodes > 0:
        # the CEM comparator (Table IV) on the first cem_episodes scenes of each benchmark,
        # at the AM loop's budget (1000 samples x 10 iterations) and at the paper's 8000 samples
        sub = [c for c in crowds if c["seed"] < cem_episodes]
        out["cem"] = {"episodes": len(sub), "planned": "one episode at a time, warm mean from the previous plan"}
        for name, kw in (("samples_1000_iters_10", dict(samples=1000, elites=100, iters=10)),
                         ("samples_8000_iters_15", dict(samples=8000, elites=800, iters=15))):
            r = M.run_cem(sub, cfg, **kw)
            row = M.summarize(r["episodes"])
            row["replan_ms"] = r["replan_ms"]
            out["cem"][name] = row
        r = M.run(sub, M.MPCConfig(batch=1000, duration=seconds))
        row = M.summarize(r["episodes"])
        row["replan_ms"] = r["replan_ms"]
        out["cem"]["am_batch_1000_same_episodes"] = row
    # the multiplier decay between steps (0.9 per step instead of the warm start's 1)
    r = M.run(crowds, M.MPCConfig(batch=1000, duration=seconds, lambda_decay=0.9))
    row = M.summarize(r["episodes"])
    row["replan_ms"] = r["replan_ms"]
    out["am_batch_1000_lambda_decay_0.9"] = row
    return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    from paper_2109_13030_b300 import workload as W
    pb = W.make_problem(WORKLOAD, 0)
    sample = 48
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; warm-up steps are not needed
    times = []
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(pb, sample, ITERS, min_seconds=0.0)
        times.append(sample * ITERS / cb["value"])
    tot = sum(times)
    value = args.steps * sample * ITERS / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "paper-shaped: B=1000, q=100, T=10 s, m=3 circles, n=10 moving ellipses, 100 AM iterations",
                       "reference": "FP64 CPU oracle (no reference code exists; the paper ships none)",
                       "sample_per_step": f"{sample} trajectories x {ITERS} iterations"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--uneven-steps", type=int, default=3)
    ap.add_argument("--precision-steps", type=int, default=3)
    ap.add_argument("--large-steps", type=int, default=3,
                    help="timed solves per kernel of the large-batch section (0 skips it)")
    ap.add_argument("--jsonl", default=None, help="also append the JSON line to this file")
    ap.add_argument("--mpc-episodes", type=int, default=0,
                    help="closed-loop episodes per crowd benchmark (0: skip; the study takes minutes)")
    ap.add_argument("--cem-episodes", type=int, default=5, help="of those, episodes per benchmark for the CEM rows")
    ap.add_argument("--mpc-seconds", type=float, default=20.0, help="closed-loop episode length (s)")
    ap.add_argument("--profile-plain", type=int, default=0, metavar="B",
                    help="profiling aid: solve 2 iterations of the paper-shaped scene at batch B with the "
                         "plain loop and exit (no JSON line)")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-plain-seconds", type=float, default=2.0)
    ap.add_argument("--detail", action="store_true",
                    help="add the full single-GPU sections (workload strings, every serving statistic) "
                         "under 'detail'; by default the line carries their short forms only")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2109_13030_b300 import trajam as TJ, workload as W

    if args.profile_plain > 0:
        pb = W.make_problem(WORKLOAD, 0, B=args.profile_plain)
        P = TJ.Problem(pb, kernel=TJ.AM_KERNEL_PLAIN)
        P.solve(torch.tensor(pb["init"], dtype=torch.float32, device="cuda"), 2,
                stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        P.close()
        return 0

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # One planning problem; its samples are split into contiguous per-rank
    # ranges of B trajectories (weak scaling), merged at the end of each step.
    from paper_2109_13030_b300 import dist_best as D
    pb_all = W.make_problem(WORKLOAD, seed=0, B=B * world)
    lo, hi = D.shard_range(B * world, rank, world)
    pb = dict(pb_all, init=pb_all["init"][lo:hi], B=hi - lo)
    # the warp-pair kernel: two warps per trajectory, no block barrier in the loop
    P = TJ.Problem(pb, kernel=TJ.AM_KERNEL_WARP)
    init_d = torch.tensor(pb["init"], dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    mind_d = torch.empty(B, dtype=torch.float32, device=dev)

    def merged_best():
        best = TJ.am_get_best(P.h)  # argmin on the device, 36 floats back
        if dist is None:
            return best
        TJ.am_get_results(P.h, mind=mind_d)
        collides = bool(mind_d[best["index"]].item() < 0.99)
        return D.merge_best(collides, best["cost"], lo + best["index"], best["coeffs"], dev)

    best_d = torch.empty(36, dtype=torch.float32, device=dev)

    def step(i=None):
        TJ.am_init_state(P.h, B, init_d, None, stream)          # cold start from resident samples
        if i is not None:
            kstarts[i].record(stream)
        TJ.am_solve_batch(P.h, B, None, None, ITERS, stream)     # the fused kernel
        if i is not None:
            kends[i].record(stream)
        TJ.am_get_best_async(P.h, best_d, stream)                # selection on the device, no host wait
        if dist is None:
            return None
        # sharded batch: the cross-rank merge on the device too (the local
        # best's collision flag from its smallest distance, one all-gather
        # of every rank's key and coefficients, the lexicographic minimum)
        TJ.am_get_results(P.h, mind=mind_d)
        collides = mind_d.index_select(0, best_d[0:1].long()) < 0.99
        return D.merge_best_device(best_d, collides, lo)

    # Host-facing measurements first, before any clock sampling: reading the
    # GPU's clocks through NVML (nvidia-smi, or the library in-process) slows
    # this process's later host-side CUDA calls severalfold on these hosts,
    # which would add to every end-to-end and latency figure below.
    # end to end through the C ABI with host buffers: pinned H2D of the
    # initial samples, the solve, D2H of per-trajectory results and the best
    init_h = torch.tensor(pb["init"], dtype=torch.float32).pin_memory()
    outs = [torch.empty(B, dtype=torch.float32).pin_memory() for _ in range(4)]
    best_h = torch.empty(36, dtype=torch.float32).pin_memory()
    # numpy views of the pinned buffers, made once
    init_np, outs_np, best_np = init_h.numpy(), [o.numpy() for o in outs], best_h.numpy()

    def e2e_step():
        TJ.am_solve_batch(P.h, B, init_np, None, ITERS, stream)
        if dist is None:
            # the selection queued behind the solve into pinned memory; the
            # results read below waits once for the solve, the status and it
            TJ.am_get_best_async(P.h, best_np, stream)
            TJ.am_get_results(P.h, *outs_np)
            if not np.isfinite(best_np[1]):
                raise RuntimeError("every trajectory of the batch is non-finite")
            return int(best_np[0])
        TJ.am_get_results(P.h, *outs_np)
        return merged_best()

    for _ in range(2):
        e2e_step()
    e2e_s = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_s.append(time.perf_counter() - t0)
    e2e_tot = sum(e2e_s)
    if dist:
        t = torch.tensor([e2e_tot], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_tot = float(t.item())
    e2e_value = world * B * ITERS * args.steps / e2e_tot

    # plain FP32 loop comparator (one launch per step), same workload
    Pp = TJ.Problem(pb, kernel=TJ.AM_KERNEL_PLAIN)
    Pp.solve(init_d, ITERS, stream=stream)
    torch.cuda.synchronize()
    plain_ms = []
    for i in range(args.plain_steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Pp.solve(init_d, ITERS, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
    plain_launches = TJ.am_last_solve_stats(Pp.h)
    plain_res = float(np.median(Pp.results()["res"]))
    Pp.close()
    # the small-tile fused kernel (block-synchronous phases, R on mma.sync), same workload
    Ps = TJ.Problem(pb, kernel=TJ.AM_KERNEL_FUSED)
    Ps.solve(init_d, ITERS, stream=stream)
    torch.cuda.synchronize()
    small_ms = []
    for i in range(args.plain_steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Ps.solve(init_d, ITERS, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        small_ms.append(e0.elapsed_time(e1))
    Ps.close()
    fused_res = float(np.median(outs[0].numpy()))

    extra = {}
    # single-GPU sections; under torchrun they would hold every rank's GPU
    # while rank 0 alone works, so they run at N = 1 only
    if rank == 0 and world == 1:
        if args.uneven_steps > 0:
            extra["uneven"] = bench_uneven(TJ, W, torch, dev, flush, args.uneven_steps)
        if args.precision_steps > 0:
            extra["precision"] = bench_precision(TJ, W, torch, dev, flush, args.precision_steps)
        if args.large_steps > 0:
            extra["large"] = bench_large(TJ, W, torch, dev, flush, args.large_steps)
        if args.serve_seconds > 0:
            extra["serving"] = bench_serving(TJ, W, args.serve_seconds, args.serve_plain_seconds)
        if args.mpc_episodes > 0:
            extra["closed_loop"] = bench_closed_loop(args.mpc_episodes, min(args.cem_episodes, args.mpc_episodes),
                                                    args.mpc_seconds)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step = 1 + TJ.am_last_solve_stats(P.h) + 1  # init state, solve, argmin

    # Timed region: CUDA events around each step on the solve's stream, and
    # around the fused kernel inside it (its average launch duration).
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kstarts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        # The clock sampler's NVML reads slow this process's host-side CUDA
        # calls severalfold, so the host would fall behind the GPU and its
        # launch gaps would enter the steps' events.  A fixed-length device
        # delay (a clock-count wait, 60 ms) ahead of the steps lets the host
        # queue all of them first; it lies outside every step's events.
        torch.cuda._sleep(int(0.06 * 2.0e9))
        for i in range(args.steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            step(i)
            ends[i].record(stream)
        torch.cuda.synchronize()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_ms = [s.elapsed_time(e) for s, e in zip(kstarts, kends)]
    tot_ms = sum(step_ms)
    if dist:
        t = torch.tensor([tot_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
        dist.barrier()
    value = world * B * ITERS * args.steps / (tot_ms / 1e3)
    kern_avg = statistics.mean(kern_ms)
    q, m, n = pb["q"], pb["m"], pb["n"]
    flops = survey_flops(q, m, n) * B * ITERS
    flops_fine = algorithmic_flops(q, m, n) * B * ITERS
    clocks = clk.summary()
    peak = peak_fp32_tflops(torch.cuda.get_device_properties(dev).multi_processor_count)
    achieved = flops / (kern_avg / 1e3) / 1e12
    achieved_fine = flops_fine / (kern_avg / 1e3) / 1e12

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper-shaped: B=1000/GPU, q=100 over 10 s, degree-10 Bernstein, m=3 circles, "
                                   "10 moving ellipses, 100 AM iterations, rho=1, then the best selection",
                       "parallelism": (f"batch of {B * world} sharded x{world}; best-key all-gather per step"
                                       if world > 1 else "single GPU"),
                       "l2": "512 MiB buffer rewritten between timed steps",
                       "kernel": "warp-pair fused persistent (two warps per trajectory), 1 launch per solve"},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": measured_traffic(),
                         "kernel": "am_warp_kernel", "kernel_ms": kern_avg, "flops_per_launch": flops,
                         "flops_basis": "scope-table figure, 130.2 kflop per trajectory-iteration",
                         "frac_finer_count": achieved_fine / peak,
                         "peak_basis": "derived FP32 peak: SMs x 128 lanes x 2 x 2032 MHz"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * 33 * 4,
                    "d2h_bytes_per_step": B * 4 * 4 + 36 * 4},
            "clocks": clocks,
        }
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(pb, B, ITERS)
        line["plain_fp32_loop"] = {"value": B * ITERS / (statistics.mean(plain_ms) / 1e3),
                                   "ms": statistics.mean(plain_ms), "launches": plain_launches,
                                   "res_median": plain_res}
        line["fused_res_median"] = fused_res
        line["small_tile_kernel"] = {"value": B * ITERS / (statistics.mean(small_ms) / 1e3),
                                     "ms": statistics.mean(small_ms)}
        line.update(summary_sections(extra))
        if "closed_loop" in extra:
            line["closed_loop"] = extra.pop("closed_loop")
        if args.detail:
            line["detail"] = extra
        line = compact(line)
        print(json.dumps(line), flush=True)
        if args.jsonl:
            with open(args.jsonl, "a") as f:
                f.write(json.dumps(dict(line, seed=0, when=time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()))) + "\n")
    P.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
