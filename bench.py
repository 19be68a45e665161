#!/usr/bin/env python
"""Throughput benchmark: degree-6 complex polynomials rooted and binned per second.

Workload: the 2^26 Littlewood-type polynomials (a_0..a_6 i.i.d. in {1,-1,i,-i},
SplitMix64 seed 2), complex64 coefficient-major, resident in HBM (3.76 GB per
step, larger than the 129 MB L2, so no L2 flush is needed between steps),
rooted by single-shift QR on the 6x6 companion matrix and binned into a
1920x1080 uint32 histogram over [-2,2]x[-1.125,1.125].

One step = clear the histogram and counters + one fused roots+density launch
over the whole batch. The headline ``value`` is the mixed mode (FP32 sweeps,
3 FP64 Newton steps, FP64 residual check); the plain FP64 GPU path is timed on
the same batch and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank solves its own 2^26 polynomials (weak
scaling), the per-rank histograms are summed once after the timed region, and
the time is the maximum over ranks. ``--impl reference`` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "deg-6 complex polys rooted+binned/s, mixed vs plain FP64, ≤1e-9 err; % of peak"
UNIT = "polys/s"
SEED = 2
DEGREE = 6
WINDOW = (-2.0, 2.0, -1.125, 1.125)
W_PIX, H_PIX = 1920, 1080
E2E_CHUNK_LOG2 = 22
# ncu summary of each form of the headline kernel, with the source hash it was taken on
PROFILE_SUMMARY = {"one_role": os.path.join(ROOT, "profiles", "solve_mixed_littlewood_deg6.md"),
                   "ws": os.path.join(ROOT, "profiles", "solve_ws_littlewood_deg6.md")}
# Each solve kernel's code and its launch (the .cu files only dispatch to them); an ncu
# traffic figure is valid only for the source it was taken on.
KERNEL_SOURCES = {"one_role": ["paper_2507_02164_gb300/csrc/rd_solve.cuh", "paper_2507_02164_gb300/csrc/rd_common.cuh",
                               "paper_2507_02164_gb300/csrc/rd_solve_launch.cuh"],
                  "ws": ["paper_2507_02164_gb300/csrc/rd_solve.cuh", "paper_2507_02164_gb300/csrc/rd_common.cuh",
                         "paper_2507_02164_gb300/csrc/rd_solve_ws.cuh"]}  # device code; launch: rd_solve_ws_launch.cuh
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (4 SMSPs x 32)
FP64_FMA_PER_SM_CLK = 2   # FP64 FMA per SM per clock: 1.25 TFLOP/s / (152 SMs x 2 flop x 2.07 GHz)


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["littlewood", "uneven", "paper", "pipeline", "adjoint"],
                    default="littlewood",
                    help="littlewood: the 2^26 degree-6 batch of the metric; uneven: 2^24 polynomials of "
                         "degree 2..12 (complex Gaussian, seed 3) in one CUDA-graph replay per step")
    ap.add_argument("--log2n", type=int, default=None, help="polynomials per GPU = 2^log2n")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the short runs of the batching, differentiation and pipeline configurations")
    return ap.parse_args(argv)


def kernel_source_hash(form: str = "one_role") -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[form]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(form: str = "one_role"):
    """Per-launch DRAM bytes of the solve kernel (form "one_role" or "ws") from
    the committed ncu summary, or None when the summary is missing or was
    taken on other kernel source."""
    try:
        text = open(PROFILE_SUMMARY[form]).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_source_hash(form):
        return None
    return float(m.group(1))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every interval_ms (default 200) while running (the
    timed region)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 200):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        load = [v for v in sm if smax and v >= 0.3 * smax] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ------------------------------------------------------ measured ALU peaks

_PEAKS = {}


def measured_alu_peaks(torch, dev, local_rank: int):
    """FP32 (FFMA) and FP64 (DFMA) throughput of this GPU, measured once per
    process with the library's probe kernel (rd_alu_peak: independent FMA
    chains on every SM), best of 5 launches of about 50 ms each, CUDA events
    on the launching stream, clocks sampled meanwhile. These are the
    denominators of the ALU roofline."""
    if "v" in _PEAKS:
        return _PEAKS["v"]
    from paper_2507_02164_gb300 import api
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    with ClockSampler(local_rank) as clk:
        for kind, iters in (("fp32", 50000), ("fp64", 1500)):
            api.alu_peak(kind, iters // 10, sink=sink)  # warm-up
            rates = []
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fl = api.alu_peak(kind, iters, sink=sink)
                e1.record(stream)
                torch.cuda.synchronize()
                rates.append(fl / (e0.elapsed_time(e1) * 1e-3))
            res[kind] = (max(rates), statistics.median(rates), fl)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    c = clk.summary()
    mhz = c.get("sm_max_mhz") or 2070.0
    _PEAKS["v"] = {
        "fp32_tflops": res["fp32"][0] / 1e12, "fp64_tflops": res["fp64"][0] / 1e12,
        "fp32_tflops_median": res["fp32"][1] / 1e12, "fp64_tflops_median": res["fp64"][1] / 1e12,
        "derived_fp32_tflops": sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12,
        "derived_fp64_tflops": sms * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12,
        "flops_per_launch": {"fp32": res["fp32"][2], "fp64": res["fp64"][2]},
        "clocks": c,
        "how": "rd_alu_peak: 4 CTAs x 256 threads per SM, 8 independent FMA chains per thread (FP32: packed "
               "fma.rn.f32x2 pairs), best of 5 launches of ~50 ms (CUDA events); derived = SMs x lanes x 2 flop "
               "x max SM clock",
    }
    return _PEAKS["v"]


def roofline_peaks(torch, dev, local_rank: int):
    """(FP32 peak, FP64 peak) in flop/s and the source line for the roofline."""
    pk = measured_alu_peaks(torch, dev, local_rank)
    src = (f"measured: rd_alu_peak FFMA {pk['fp32_tflops']:.2f} / DFMA {pk['fp64_tflops']:.3f} TFLOP/s "
           f"(best of 5; derived {pk['derived_fp32_tflops']:.1f} / {pk['derived_fp64_tflops']:.3f})")
    return pk["fp32_tflops"] * 1e12, pk["fp64_tflops"] * 1e12, src


# ------------------------------------------------------------- CPU oracle

def cpu_oracle_rate(seconds: float, start_index: int = 0, first_idx=None):
    """Oracle solve + histogram on the host cores for about `seconds`; returns
    (polys/s, threads used, polys done, first chunk). The first chunk is the
    polynomials first_idx when given (their oracle roots and status are
    returned with their coefficients, for the root-error report), then
    chunks of 65,536 consecutive polynomials of the stream."""
    import numpy as np

    import oracle
    from paper_2507_02164_gb300 import workloads as WL
    oracle.build()
    chunk = 1 << 16
    done, elapsed, threads, k = 0, 0.0, 0, 0
    first = None
    while elapsed < seconds or first is None:
        if first is None and first_idx is not None:
            idx = np.asarray(first_idx, dtype=np.uint64)
        else:
            idx = np.arange(start_index + k * chunk, start_index + (k + 1) * chunk, dtype=np.uint64)
            k += 1
        co = WL.littlewood(SEED, idx).astype(np.complex128)
        t0 = time.perf_counter()
        roots, status, _, threads = oracle.solve(co, tol=1e-13)
        oracle.hist(roots, WINDOW, W_PIX, H_PIX)
        elapsed += time.perf_counter() - t0
        done += idx.size
        if first is None:
            first = (co, roots, status)
    return done / elapsed, threads, done, first


def run_reference(args, rank: int):
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2507_02164_gb300 import workloads as WL
    oracle.build()
    S = 1 << 18
    times = []
    threads = 0
    for step in range(args.warmup + args.steps):
        idx = np.arange(step * S, (step + 1) * S, dtype=np.uint64)
        co = WL.littlewood(SEED, idx).astype(np.complex128)
        t0 = time.perf_counter()
        roots, _, _, threads = oracle.solve(co, tol=1e-13)
        oracle.hist(roots, WINDOW, W_PIX, H_PIX)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = S * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded Littlewood {1,-1,i,-i} degree-6 polynomials (SplitMix64 seed 2)",
        "config": workload_config(args, args.gpus, ref_sample=S),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{S} polynomials per step (indices step*{S}..), FP64 oracle solve + histogram, "
                                   f"OpenMP over {threads} host threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, world: int, ref_sample=None):
    cfg = {
        "workload": f"littlewood-deg6-2^{args.log2n}: a_k in {{1,-1,i,-i}} complex64, fused roots + "
                    f"{W_PIX}x{H_PIX} uint32 histogram over [-2,2]x[-1.125,1.125]",
        "polys_per_gpu": 1 << args.log2n,
        "degree": DEGREE,
        "mixed": "FP32 QR sweeps (Wilkinson shift, deflation 4*2^-24, <=40 sweeps/root) + 3 FP64 Newton steps "
                 "+ FP64 residual/separation check",
        "plain": "FP64 QR sweeps (Wilkinson shift, deflation 1e-13, <=40 sweeps/root)",
        "l2_flush": "inputs larger than L2 (3.76 GB of coefficients per GPU per step)",
        "parallelism": f"dp{world}",
    }
    if ref_sample:
        cfg["reference_sample_per_step"] = ref_sample
    return cfg


# ---------------------------------------------------------------- GPU leg

def match_roots(gpu, ref):
    """Reorder each row of gpu [n, d] to pair with the same row of ref: the
    nearest-root pairing where it is a permutation, else the assignment of
    least total distance (rows where roots lie closer together than their
    errors)."""
    import numpy as np
    from scipy.optimize import linear_sum_assignment
    dist = np.abs(gpu[:, None, :] - ref[:, :, None])  # [n, ref j, gpu k]
    near = dist.argmin(axis=2)
    ok = np.all(np.sort(near, axis=1) == np.arange(ref.shape[1])[None, :], axis=1)
    out = np.take_along_axis(gpu, near, axis=1)
    for i in np.nonzero(~ok)[0]:
        rows, cols = linear_sum_assignment(np.nan_to_num(dist[i], nan=1e300, posinf=1e300))
        out[i, rows] = gpu[i, cols]
    return out


# Every root, however ill-conditioned, is held to KAPPA_SCALED * max(1, kappa)
# (the oracle's own deflation at 1e-13 leaves about 10 kappa 1e-13), and the
# roots left out of the plain bar (kappa above the cap) must stay a small
# share of those compared: the bar the parity tests apply.
KAPPA_SCALED = 1e-11
MAX_EXCLUDED = 0.06


def root_error_summary(gpu, status, ref, ref_status, coeffs, bar, kappa_cap):
    """Relative error |z - z_ref| / max(1, |z_ref|) of matched roots where
    both solvers report OK. Roots with condition number above kappa_cap (the FP64 reference
    itself is not accurate to the bar there) are reported apart; within_bar
    needs the bar on the others, KAPPA_SCALED * max(1, kappa) on every root,
    and at most MAX_EXCLUDED of the roots apart. kappa =
    sum |a_k| |z|^k / (max(1, |z|) |p'(z)|), the oracle's definition."""
    import numpy as np
    ok = (status == 0) & (ref_status == 0)
    g = match_roots(gpu[ok], ref[ok])
    r, a = ref[ok], coeffs[ok]
    err = np.abs(g - r) / np.maximum(1.0, np.abs(r))
    d = a.shape[1] - 1
    az = np.abs(r)
    num = sum(np.abs(a[:, k:k + 1]) * az ** k for k in range(d + 1))
    dp = sum(k * a[:, k:k + 1] * r ** (k - 1) for k in range(1, d + 1))
    with np.errstate(divide="ignore", invalid="ignore"):
        # the condition number of the error measure |dz| / max(1, |z|), as the
        # oracle (or_root_condition) and the parity tests define it
        kappa = num / (np.maximum(az, 1.0) * np.abs(dp))
    well = kappa <= kappa_cap
    kappa_ok = bool(np.all(err <= np.maximum(bar, KAPPA_SCALED * np.maximum(1.0, np.nan_to_num(kappa, nan=np.inf)))))
    excluded = float((~well).mean()) if well.size else 0.0
    max_well = float(err[well].max(initial=0.0))
    return {"max_rel_err": max_well, "median_rel_err": float(np.median(err[well])) if well.any() else 0.0,
            "roots_compared": int(well.sum()), "bar": bar,
            "within_bar": bool(max_well <= bar and kappa_ok and excluded <= MAX_EXCLUDED),
            "kappa_scaled_ok": kappa_ok, "excluded_fraction": excluded, "max_excluded_fraction": MAX_EXCLUDED,
            "ill_conditioned_roots": int((~well).sum()), "ill_conditioned_max_rel_err":
            float(err[~well].max(initial=0.0)), "kappa_cap": kappa_cap,
            "status_counts": np.bincount(status, minlength=4).tolist()}


def algorithmic_flops(st: dict):
    """(FP32 flops, FP64 flops) of the counted launches, as the kernel counted
    them (rd_stats flops_fp32 / flops_fp64; convention in include/rootdensity.h:
    20 flop per rotated pair, 24 per Givens pair, 60 per sweep in the sweep
    precision; 8d+2 FP64 + 8d+3 FP32 per Newton step; 8d+4 FP64 + 2d+4 FP32
    per polished root; 4 FP64 per binned root in the plain mode)."""
    return float(st["flops_fp32"]), float(st["flops_fp64"])


def run_ours(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2507_02164_gb300 import api, build, dist as D, workloads as WL

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = 1 << args.log2n
    start, _ = D.shard_range(n, rank)
    coeffs = WL.littlewood_soa_torch(SEED, start, n, dev)
    win = api.Window(*WINDOW)
    hist = api.new_hist(W_PIX, H_PIX, dev)
    stats = api.new_stats(dev)
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2507_02164_gb300 import autotune
    tuned = {m: autotune.tune(m, degrees=[DEGREE]) for m in ("mixed",) + (() if args.no_plain else ("plain",))}

    def timed_leg(mode: str, **overrides):
        p = autotune.degree_params(tuned[mode], DEGREE, mode)
        for k, v in overrides.items():
            setattr(p, k, v)
        k_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        k_end = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        for _ in range(args.warmup):
            api.hist_clear(hist)
            api.hist_clear(stats)
            api.roots_density(coeffs, win, hist, mode=mode, params_=p, stats=stats)
        barrier()
        with ClockSampler(local_rank) as clk:
            t0.record(stream)
            for s in range(args.steps):
                api.hist_clear(hist)
                api.hist_clear(stats)
                k_start[s].record(stream)
                api.roots_density(coeffs, win, hist, mode=mode, params_=p, stats=stats)
                k_end[s].record(stream)
            t1.record(stream)
            torch.cuda.synchronize()
        elapsed_ms = D.max_over_ranks(t0.elapsed_time(t1), device=dev)
        kern_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(k_start, k_end))
        st = api.stats_dict(stats)
        return elapsed_ms, kern_ms, st, clk.summary()

    # the roofline's denominators, measured on this GPU before the timed legs
    alu_peaks = measured_alu_peaks(torch, dev, local_rank)

    elapsed_mx, kern_mx, st_mx, clk_mx = timed_leg("mixed")
    launches_per_step = 3  # histogram clear, counter clear, fused solve
    polys_total = n * world * args.steps
    value = polys_total / (elapsed_mx * 1e-3)

    # ---- end to end from pinned host memory through the public API, right
    # after the device-resident leg (before the slower comparison legs)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, coeffs, win, dev, world, autotune.degree_params(tuned["mixed"], DEGREE, "mixed"))

    # the same batch with every warp sweeping and then polishing its own
    # polynomials (the fastest such shape), and the double-float polish
    # variant, which has only that form (neither is the headline)
    one = tuned["mixed"]["degrees"][str(DEGREE)]["one_role"]
    one_shape = dict(block=one["block"], ctas_per_sm=one["ctas_per_sm"], lanes=one["lanes"], polish_warps=0)
    elapsed_or, kern_or, st_or, clk_or = timed_leg("mixed", **one_shape)
    # the FP32-pipe compensated polish (RD_POLISH_DF) in the launch shape the
    # tuner picks for it (warp-specialised or not)
    tuned_df = autotune.tune("mixed", degrees=[DEGREE], polish="df")
    df_e = tuned_df["degrees"][str(DEGREE)]
    df_shape = dict(block=df_e["block"], ctas_per_sm=df_e["ctas_per_sm"], lanes=df_e["lanes"],
                    polish_warps=df_e.get("polish_warps", 0), polish_mode=api.N.POLISH_DF)
    elapsed_df, kern_df, st_df, clk_df = timed_leg("mixed", **df_shape)

    plain = None
    if not args.no_plain:
        elapsed_pl, kern_pl, st_pl, clk_pl = timed_leg("plain")
        plain = {"elapsed_ms": elapsed_pl, "kern_ms": kern_pl, "stats": st_pl, "clocks": clk_pl}

    # the small plain-FP64 configuration's latency: 65,536 monic degree-6
    # polynomials with seeded roots in the unit disk (complex128), roots +
    # histogram over [-1.5,1.5]x[-0.84375,0.84375], one CUDA-graph replay per
    # call, median of 20 after 3 warm-ups
    latency = small_batch_latency(api, WL, torch, dev, stream) if rank == 0 else None

    # the root-error subsample i = 1024 k of this batch, solved again by each GPU
    # path with its timed launch shape (a polynomial's roots do not depend on
    # its neighbours in the batch); compared with the oracle in the CPU leg
    sub_idx, sub_roots = None, {}
    if rank == 0 and not args.no_cpu and n >= 1024:
        import numpy as np
        sub_idx = np.arange(min(1 << 16, n // 1024), dtype=np.int64) * 1024
        sub = coeffs[:, torch.from_numpy(sub_idx).to(dev)].contiguous()
        for mode in tuned:
            r, stt = api.roots_batched(sub, mode=mode, params_=autotune.degree_params(tuned[mode], DEGREE, mode))
            sub_roots[mode] = (r.cpu().numpy().T, stt.cpu().numpy())
        r, stt = api.roots_batched(sub, mode="mixed", params_=autotune.degree_params(tuned_df, DEGREE, "mixed", "df"))
        sub_roots["mixed_df"] = (r.cpu().numpy().T, stt.cpu().numpy())

    # one exchange step: sum the per-rank images (after the timed region)
    reduce_ms = None
    if world > 1:
        torch.cuda.synchronize()
        t = time.perf_counter()
        D.reduce_images(hist, dst=0)
        torch.cuda.synchronize()
        reduce_ms = 1e3 * (time.perf_counter() - t)


    if rank != 0:
        return
    p32, p64, peak_src = roofline_peaks(torch, dev, local_rank)
    f32, f64 = algorithmic_flops(st_mx)
    t_k = kern_mx * 1e-3
    frac32, frac64 = f32 / p32 / t_k, f64 / p64 / t_k
    traffic = profiled_traffic("ws" if tuned["mixed"]["degrees"][str(DEGREE)].get("polish_warps", 0) else "one_role")
    pw = tuned["mixed"]["degrees"][str(DEGREE)].get("polish_warps", 0)
    blk = tuned["mixed"]["degrees"][str(DEGREE)]["block"]
    kernel_name = (f"rd::solve_ws_kernel<6, float2> (warp-specialised: {pw} polish warps of {blk // 32})" if pw
                   else "rd::solve_kernel<6, float, float2, MIXED>")
    roofline = {
        "bound": "alu", "kernel": kernel_name,
        "achieved": (f32 + f64 * p32 / p64) / t_k / 1e12, "peak": p32 / 1e12, "unit": "TFLOP/s",
        "frac": frac32 + frac64, "traffic": traffic,
        "note": "FP32-equivalent: FP64 flops weighted by the FP32/FP64 peak ratio; frac = fp32_frac + fp64_frac",
        "fp32_frac": frac32, "fp64_frac": frac64,
        "fp32_tflops": f32 / t_k / 1e12, "fp64_tflops": f64 / t_k / 1e12,
        "peak_fp32_tflops": p32 / 1e12, "peak_fp64_tflops": p64 / 1e12,
        "peak_source": peak_src,
        "kernel_ms": kern_mx,
        "algorithmic_flops_per_launch": {"fp32": f32, "fp64": f64},
    }
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_mx / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic: seeded Littlewood {1,-1,i,-i} degree-6 polynomials (SplitMix64 seed 2), generated on device",
        "config": dict(workload_config(args, world), launch_shapes={m: tuned[m]["degrees"][str(DEGREE)] for m in tuned}),
        "roofline": roofline,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk_mx,
        "alu_peaks": alu_peaks,
        "mixed": {"status": {k: st_mx[k] for k in ("status_ok", "status_not_converged", "status_rejected",
                                                   "status_degenerate")},
                  "sweeps_per_poly": st_mx["sweeps"] / max(1, st_mx["polys"]),
                  "binned": st_mx["binned"], "out_of_window": st_mx["out_of_window"],
                  "paper_equiv_gflops": value * 41.9e3 / 1e9,
                  "equiv_qr_sweeps_per_s": value * st_mx["sweeps"] / max(1, st_mx["polys"])},
    }
    o32, o64 = algorithmic_flops(st_or)
    line["mixed_one_role"] = {
        "value": polys_total / (elapsed_or * 1e-3), "unit": UNIT, "ms_per_step": elapsed_or / args.steps,
        "kernel_ms": kern_or, "fp32_frac": o32 / p32 / (kern_or * 1e-3), "fp64_frac": o64 / p64 / (kern_or * 1e-3),
        "shape": one_shape, "identical_histogram_counters": st_or == st_mx,
        "note": "rd::solve_kernel: every warp sweeps and then polishes its own 32 polynomials", "clocks": clk_or}
    g32, g64 = algorithmic_flops(st_df)
    t_df = kern_df * 1e-3
    line["mixed_df_polish"] = {
        "value": polys_total / (elapsed_df * 1e-3), "unit": UNIT, "ms_per_step": elapsed_df / args.steps,
        "kernel_ms": kern_df, "fp32_frac": g32 / p32 / t_df, "fp64_frac": g64 / p64 / t_df,
        "frac": g32 / p32 / t_df + g64 / p64 / t_df,
        "fp32_tflops": g32 / t_df / 1e12, "fp64_tflops": g64 / t_df / 1e12,
        "shape": {k: v for k, v in df_shape.items() if k != "polish_mode"}, "tuned_ms": df_e["ms"],
        "status": {k: st_df[k] for k in ("status_ok", "status_not_converged", "status_rejected", "status_degenerate")},
        "newton_steps_per_poly": st_df["newton_steps"] / max(1, st_df["polys"]),
        "over_fp64_polish": kern_mx / kern_df,
        "note": "RD_POLISH_DF: 3 Newton steps on the FP32 pipe (z as a float pair, p(z) by the compensated "
                "Horner scheme), FP64 final residual check; sweep warps and polish warps as the tuner picked",
        "clocks": clk_df}
    if plain is not None:
        pv = polys_total / (plain["elapsed_ms"] * 1e-3)
        _, g64 = algorithmic_flops(plain["stats"])
        line["plain_fp64"] = {
            "value": pv, "unit": UNIT, "ms_per_step": plain["elapsed_ms"] / args.steps,
            "kernel_ms": plain["kern_ms"], "fp64_frac": g64 / p64 / (plain["kern_ms"] * 1e-3),
            "fp64_tflops": g64 / (plain["kern_ms"] * 1e-3) / 1e12,
            "sweeps_per_poly": plain["stats"]["sweeps"] / max(1, plain["stats"]["polys"]),
            "status_not_converged": plain["stats"]["status_not_converged"], "clocks": plain["clocks"]}
        line["mixed_over_plain"] = value / pv
    if e2e is not None:
        line["e2e"] = e2e
    if latency is not None:
        line["small_batch_latency"] = latency
    if reduce_ms is not None:
        line["hist_reduce_ms"] = reduce_ms
    if not args.no_cpu:
        v, threads, done, (co_s, ref_s, ref_st) = cpu_oracle_rate(args.cpu_seconds, first_idx=sub_idx)
        first = f"the {sub_idx.size} polynomials i = 1024 k, then " if sub_idx is not None else ""
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{done} polynomials of the same Littlewood stream: {first}the first ones "
                                          f"in chunks of 65536; FP64 oracle solve (tol 1e-13) + histogram, "
                                          f"~{args.cpu_seconds:.0f} s"}
        # root error of the GPU paths on that subsample (the oracle's first chunk)
        if sub_idx is not None:
            line["root_error"] = {
                "subsample": f"the {sub_idx.size} polynomials i = 1024 k of the batch, GPU roots vs the FP64 "
                             "oracle (tol 1e-13), matched per polynomial; error |z - z_oracle| / max(1, |z_oracle|)",
                "mixed": root_error_summary(sub_roots["mixed"][0], sub_roots["mixed"][1], ref_s, ref_st, co_s,
                                            1e-9, 1e3),
            }
            if "plain" in sub_roots:
                line["root_error"]["plain_fp64"] = root_error_summary(sub_roots["plain"][0], sub_roots["plain"][1],
                                                                      ref_s, ref_st, co_s, 1e-11, 1e2)
            line["root_error"]["mixed_df_polish"] = root_error_summary(
                sub_roots["mixed_df"][0], sub_roots["mixed_df"][1], ref_s, ref_st, co_s, 1e-9, 1e3)
    if world == 1 and not args.no_configs:
        line["configs"] = other_configs(args, rank, world, local_rank)
    print(json.dumps(line), flush=True)


def _compact(line: dict, extra=()) -> dict:
    keys = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype", "roofline", "clocks",
            "cpu_baseline", "root_error", "gpu_launches") + tuple(extra)
    out = {k: line[k] for k in keys if k in line}
    out["workload"] = line["config"]["workload"]
    return out


def other_configs(args, rank, world, local_rank) -> dict:
    """The batching, differentiation and full-pipeline configurations, each
    on a short run (at most 5 timed steps after 3 warm-ups, its own clocks,
    roofline against the measured peaks and an oracle baseline of ~4 s on
    the host cores); the full runs are bench.py --workload uneven | adjoint |
    pipeline."""
    import copy
    sub = copy.copy(args)
    sub.steps, sub.warmup = min(args.steps, 5), 3
    sub.cpu_seconds, sub.no_e2e = min(args.cpu_seconds, 4.0), True
    sub.min_timed_s = 0.5  # at least 0.5 s of timed work, so the clock sampler sees it
    t0 = time.perf_counter()
    out = {}
    u = copy.copy(sub)
    u.log2n = 24
    out["batching"] = _compact(run_uneven(u, rank, world, local_rank, emit=False),
                               ("status", "sweeps_per_poly", "mixed_df_polish"))
    out["differentiation"] = _compact(run_adjoint(sub, rank, world, local_rank, emit=False),
                                      ("c128", "c64", "grad_error"))
    out["full_pipeline"] = _compact(run_pipeline(sub, rank, world, local_rank, emit=False),
                                    ("l2_approx_ms", "roots_density_ms", "roots_roofline", "fused", "kept_roots",
                                     "status"))
    out["seconds"] = time.perf_counter() - t0
    return out


def bind_to_gpu_local_cpus(torch, dev):
    """Restrict this process to the CPUs the kernel lists as local to the GPU
    (sysfs local_cpulist of its PCI function), so that page-locked buffers
    allocated next land on the memory node next to it (the caller restores
    the previous set afterwards). Best effort: returns what was done, or why
    not."""
    try:
        props = torch.cuda.get_device_properties(dev)
        bdf = f"{props.pci_domain_id:04x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bdf}/local_cpulist") as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return {"bound": False, "why": f"no allowed CPU in {spec}", "pci": bdf}
        before = os.sched_getaffinity(0)
        os.sched_setaffinity(0, cpus)
        return {"bound": True, "pci": bdf, "cpus": spec, "_restore": before}
    except (OSError, AttributeError, ValueError) as e:
        return {"bound": False, "why": f"{type(e).__name__}: {e}"[:120]}


def release_pinned(torch):
    """Return cached page-locked host memory and device blocks to the system."""
    import gc
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    try:
        torch._C._host_emptyCache()
    except AttributeError:
        pass


def run_e2e(args, coeffs_dev, win, dev, world, p):
    """Same metric through the public API with the inputs in page-locked host
    memory: each step, rd_roots_density (launch shape p) reads the 56 B of
    every polynomial straight from host memory across the host link while it
    solves (the buffer is mapped into the device address space; zero copy),
    then the histogram and counters are read back to the host. The chunked
    variant with explicit copies on a copy stream is measured beside it."""
    import torch

    from paper_2507_02164_gb300 import api, dist as D

    n = coeffs_dev.shape[1]
    affinity = bind_to_gpu_local_cpus(torch, dev)
    host = coeffs_dev.cpu().pin_memory()
    if "_restore" in affinity:
        os.sched_setaffinity(0, affinity.pop("_restore"))
    hist = api.new_hist(W_PIX, H_PIX, dev)
    stats = api.new_stats(dev)
    hist_h = torch.empty_like(hist, device="cpu").pin_memory()
    stats_h = torch.empty_like(stats, device="cpu").pin_memory()
    comp = torch.cuda.current_stream()

    def step():
        api.hist_clear(hist)
        api.hist_clear(stats)
        api.roots_density(host, win, hist, mode="mixed", params_=p, stats=stats)
        hist_h.copy_(hist, non_blocking=True)
        stats_h.copy_(stats, non_blocking=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index or 0) as clk:
        t0.record(comp)
        for _ in range(args.steps):
            step()
        t1.record(comp)
        torch.cuda.synchronize()
    ms = D.max_over_ranks(t0.elapsed_time(t1), device=dev)
    h2d = host.numel() * host.element_size()
    d2h = hist_h.numel() * hist_h.element_size() + stats_h.numel() * stats_h.element_size()
    out = {"value": n * world * args.steps / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": ms / args.steps, "gpu_launches_per_step": 3,
           "input": "page-locked host memory, read by the solve kernel across the host link (zero copy)",
           "host_link_gbs_needed": h2d / (ms / args.steps * 1e-3) / 1e9, "host_affinity": affinity,
           "clocks": clk.summary()}
    del host
    release_pinned(torch)
    out["copy_engine"] = run_e2e_copies(args, coeffs_dev, win, dev, world, p)
    return out


def run_e2e_copies(args, coeffs_dev, win, dev, world, p):
    """Same metric through the public API with the inputs in pinned host memory:
    per step, the chunks are copied host-to-device on a copy stream while the
    previous chunk is solved, and the histogram and counters are read back."""
    import torch

    from paper_2507_02164_gb300 import api

    n = coeffs_dev.shape[1]
    chunk = min(n, 1 << E2E_CHUNK_LOG2)
    nchunks = (n + chunk - 1) // chunk
    affinity = bind_to_gpu_local_cpus(torch, dev)  # page-locked buffers on the GPU's own memory node
    host = []
    for c in range(nchunks):
        part = coeffs_dev[:, c * chunk:(c + 1) * chunk].contiguous().cpu().pin_memory()
        host.append(part)
    if "_restore" in affinity:  # the pages are placed; give the CPUs back to the other legs
        os.sched_setaffinity(0, affinity.pop("_restore"))
    bufs = [torch.empty((DEGREE + 1) * chunk, dtype=torch.complex64, device=dev) for _ in range(2)]
    hist = api.new_hist(W_PIX, H_PIX, dev)
    stats = api.new_stats(dev)
    hist_h = torch.empty_like(hist, device="cpu").pin_memory()
    stats_h = torch.empty_like(stats, device="cpu").pin_memory()
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream(device=dev)
    freed = [torch.cuda.Event() for _ in range(2)]
    loaded = [torch.cuda.Event() for _ in range(2)]

    def step():
        api.hist_clear(hist)
        api.hist_clear(stats)
        start_ev = torch.cuda.Event()
        start_ev.record(comp)
        copy.wait_event(start_ev)
        for c in range(nchunks):
            b = c % 2
            m = host[c].shape[1]
            dst = bufs[b][:(DEGREE + 1) * m].view(DEGREE + 1, m)  # contiguous [d+1, m]
            with torch.cuda.stream(copy):
                if c >= 2:
                    copy.wait_event(freed[b])
                dst.copy_(host[c], non_blocking=True)
                loaded[b].record(copy)
            comp.wait_event(loaded[b])
            api.roots_density(dst, win, hist, mode="mixed", params_=p, stats=stats)
            freed[b].record(comp)
        hist_h.copy_(hist, non_blocking=True)
        stats_h.copy_(stats, non_blocking=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index or 0) as clk:
        t0.record(comp)
        for _ in range(args.steps):
            step()
        t1.record(comp)
        torch.cuda.synchronize()
    from paper_2507_02164_gb300 import dist as D
    ms = D.max_over_ranks(t0.elapsed_time(t1), device=dev)
    h2d = sum(h.numel() * h.element_size() for h in host)
    e2e_clocks = clk.summary()
    d2h = hist_h.numel() * hist_h.element_size() + stats_h.numel() * stats_h.element_size()
    # the copies alone, for reference: host-to-device bandwidth of this machine
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(comp)
    for c in range(nchunks):
        m = host[c].shape[1]
        bufs[c % 2][:(DEGREE + 1) * m].view(DEGREE + 1, m).copy_(host[c], non_blocking=True)
    c1.record(comp)
    torch.cuda.synchronize()
    h2d_gbs = h2d / (c0.elapsed_time(c1) * 1e-3) / 1e9
    # release the pinned staging buffers now (3.76 GB of page-locked host memory)
    del host, bufs
    release_pinned(torch)
    return {"value": n * world * args.steps / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms / args.steps, "chunks_per_step": nchunks,
            "gpu_launches_per_step": 2 + nchunks, "h2d_copy_only_gbs": h2d_gbs, "host_affinity": affinity,
            "clocks": e2e_clocks}


UNEVEN_SEED = 3
UNEVEN_WINDOW = (-3.0, 3.0, -1.6875, 1.6875)
UNEVEN_METRIC = "uneven-degree (2..12) complex polys rooted+binned/s, mixed, one CUDA-graph replay per step"


def cpu_oracle_rate_uneven(seconds: float):
    """Oracle solve + histogram of the uneven stream on the host cores for about
    `seconds`; returns (polys/s, threads, polys done, first chunk) with the
    first chunk's {degree: (polynomial indices, coefficients, roots, status)}."""
    import numpy as np

    import oracle
    from paper_2507_02164_gb300 import workloads as WL
    oracle.build()
    chunk = 1 << 15
    done, elapsed, threads, k = 0, 0.0, 0, 0
    while elapsed < seconds:
        idx = np.arange(k * chunk, (k + 1) * chunk, dtype=np.uint64)
        packed, deg, off = WL.uneven_gaussian(UNEVEN_SEED, idx)
        packed = packed.astype(np.complex128)
        rows_by_deg = {}
        for d in range(2, 13):
            sel = np.nonzero(deg == d)[0]
            if sel.size:
                rows_by_deg[d] = packed[(off[sel][:, None] + np.arange(d + 1)[None, :])]
        t0 = time.perf_counter()
        solved = {}
        for d, rows in rows_by_deg.items():
            roots, status, _, threads = oracle.solve(rows, tol=1e-13)
            oracle.hist(roots, UNEVEN_WINDOW, W_PIX, H_PIX)
            solved[d] = (roots, status)
        elapsed += time.perf_counter() - t0
        if k == 0:
            first = {d: (np.nonzero(deg == d)[0], rows_by_deg[d], r, st) for d, (r, st) in solved.items()}
        done += chunk
        k += 1
    return done / elapsed, threads, done, first


def run_uneven(args, rank: int, world: int, local_rank: int, emit: bool = True):
    import torch

    from paper_2507_02164_gb300 import api, build, dist as D, workloads as WL

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = 1 << args.log2n
    start, _ = D.shard_range(n, rank)
    packed, deg, off = WL.uneven_gaussian_torch(UNEVEN_SEED, start, n, dev)
    ws = api.new_uneven_workspace(n, packed.numel(), torch.complex64, dev)
    win = api.Window(*UNEVEN_WINDOW)
    hist = api.new_hist(W_PIX, H_PIX, dev)
    stats = api.new_stats(dev)
    p = api.params("mixed")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    from paper_2507_02164_gb300 import autotune
    tuned = autotune.tune("mixed", degrees=range(2, 13))
    tuning = autotune.uneven_tuning(tuned)

    def step_body():
        api.hist_clear(hist)
        api.hist_clear(stats)
        api.roots_uneven(packed, deg, off, ws, mode="mixed", params_=p, tuning=tuning, window=win, hist=hist,
                         stats=stats, want_roots=False, want_status=False)

    step_body()  # eager once (loads the library, sizes the grids)
    torch.cuda.synchronize()
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            step_body()
    torch.cuda.current_stream().wait_stream(side)
    launches_per_step = 2 + 16  # two clears; clear, count, scan, pack + 12 per-degree solvers
    for _ in range(args.warmup):
        graph.replay()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            graph.replay()
        t1.record(stream)
        torch.cuda.synchronize()
    ms = D.max_over_ranks(t0.elapsed_time(t1), device=dev)
    st = api.stats_dict(stats)
    value = n * world * args.steps / (ms * 1e-3)
    if world > 1:
        D.reduce_images(hist, dst=0)

    # the same batch and graph with the FP32-pipe compensated polish
    # (RD_POLISH_DF), each bin in the one-role shape the tuner picks for it
    tuned_df = autotune.tune("mixed", degrees=range(2, 13), polish="df")
    tuning_df = autotune.uneven_tuning(tuned_df)
    p_df = api.params("mixed", polish_mode="df")
    hist_df = api.new_hist(W_PIX, H_PIX, dev)
    stats_df = api.new_stats(dev)

    def step_df():
        api.hist_clear(hist_df)
        api.hist_clear(stats_df)
        api.roots_uneven(packed, deg, off, ws, mode="mixed", params_=p_df, tuning=tuning_df, window=win,
                         hist=hist_df, stats=stats_df, want_roots=False, want_status=False)

    step_df()
    torch.cuda.synchronize()
    graph_df = torch.cuda.CUDAGraph()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph_df, stream=side):
            step_df()
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(args.warmup):
        graph_df.replay()
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk_df:
        d0.record(stream)
        for _ in range(args.steps):
            graph_df.replay()
        d1.record(stream)
        torch.cuda.synchronize()
    ms_df = D.max_over_ranks(d0.elapsed_time(d1), device=dev)
    st_df = api.stats_dict(stats_df)

    # end to end: inputs in page-locked host memory. Main: the graph's own
    # kernels (count, pack) read them across the host link (zero copy);
    # beside it: explicit copies into the device buffers before each replay
    e2e = None
    if not args.no_e2e:
        hp, hd, ho = (packed.cpu().pin_memory(), deg.cpu().pin_memory(), off.cpu().pin_memory())
        hist_h = torch.empty_like(hist, device="cpu").pin_memory()
        stats_h = torch.empty_like(stats, device="cpu").pin_memory()
        h2d = hp.numel() * hp.element_size() + hd.numel() + ho.numel() * 8
        d2h = hist_h.numel() * 4 + stats_h.numel() * 8

        def host_body():
            api.hist_clear(hist)
            api.hist_clear(stats)
            api.roots_uneven(hp, hd, ho, ws, mode="mixed", params_=p, tuning=tuning, window=win, hist=hist,
                             stats=stats, want_roots=False, want_status=False)

        host_body()
        torch.cuda.synchronize()
        graph_h = torch.cuda.CUDAGraph()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph_h, stream=side):
                host_body()
        stream.wait_stream(side)

        def time_e2e(step):
            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            return D.max_over_ranks(e0.elapsed_time(e1), device=dev)

        def zero_copy_step():
            graph_h.replay()
            hist_h.copy_(hist, non_blocking=True)
            stats_h.copy_(stats, non_blocking=True)

        def copy_step():
            packed.copy_(hp, non_blocking=True)
            deg.copy_(hd, non_blocking=True)
            off.copy_(ho, non_blocking=True)
            graph.replay()
            hist_h.copy_(hist, non_blocking=True)
            stats_h.copy_(stats, non_blocking=True)

        # pipelined: the batch in 4 chunks of polynomials (each with its own
        # offsets, as a producer emits them), chunk c+1 copied on a copy stream
        # while chunk c is solved; one workspace, two sets of input buffers
        K = 4
        bounds = [n * k // K for k in range(K + 1)]
        off_cpu = off.cpu()
        chunks = []
        for k in range(K):
            a, b = bounds[k], bounds[k + 1]
            c0, c1 = int(off_cpu[a]), int(off_cpu[b])
            chunks.append((hp[c0:c1], hd[a:b], (off_cpu[a:b + 1] - c0).pin_memory()))
        max_c = max(c[0].numel() for c in chunks)
        max_n = max(c[1].numel() for c in chunks)
        dbuf = [(torch.empty(max_c, dtype=packed.dtype, device=dev), torch.empty(max_n, dtype=torch.uint8, device=dev),
                 torch.empty(max_n + 1, dtype=torch.int64, device=dev)) for _ in range(2)]
        copy_st = torch.cuda.Stream(device=dev)
        loaded = [torch.cuda.Event() for _ in range(2)]
        freed = [torch.cuda.Event() for _ in range(2)]

        def pipelined_step():
            api.hist_clear(hist)
            api.hist_clear(stats)
            start = torch.cuda.Event()
            start.record(stream)
            copy_st.wait_event(start)
            for k, (cp, cd, co) in enumerate(chunks):
                b = k % 2
                dc, dd, do = (dbuf[b][0][:cp.numel()], dbuf[b][1][:cd.numel()], dbuf[b][2][:co.numel()])
                with torch.cuda.stream(copy_st):
                    if k >= 2:
                        copy_st.wait_event(freed[b])
                    dc.copy_(cp, non_blocking=True)
                    dd.copy_(cd, non_blocking=True)
                    do.copy_(co, non_blocking=True)
                    loaded[b].record(copy_st)
                stream.wait_event(loaded[b])
                api.roots_uneven(dc, dd, do, ws, mode="mixed", params_=p, tuning=tuning, window=win, hist=hist,
                                 stats=stats, want_roots=False, want_status=False)
                freed[b].record(stream)
            hist_h.copy_(hist, non_blocking=True)
            stats_h.copy_(stats, non_blocking=True)

        ems = time_e2e(pipelined_step)
        st_e2e = api.stats_dict(stats)
        zms = time_e2e(zero_copy_step)
        cms = time_e2e(copy_step)
        e2e = {"value": n * world * args.steps / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ems / args.steps, "polys_solved": st_e2e["polys"],
               "input": f"page-locked host memory in {K} chunks of polynomials, each copied on a copy stream while "
                        "the previous chunk is solved (one rd_roots_uneven call per chunk)",
               "gpu_launches_per_step": 2 + 16 * K,
               "zero_copy": {"value": n * world * args.steps / (zms * 1e-3), "ms_per_step": zms / args.steps,
                             "note": "the graph's count and pack kernels read the host memory directly"},
               "copy_engine": {"value": n * world * args.steps / (cms * 1e-3), "ms_per_step": cms / args.steps,
                               "note": "explicit host-to-device copies of the whole batch before each replay"}}
    if rank != 0:
        return None
    p32, p64, peak_src = roofline_peaks(torch, dev, local_rank)
    f32, f64 = algorithmic_flops(st)
    t = ms * 1e-3 / args.steps
    line = {
        "metric": UNEVEN_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic: seeded complex-Gaussian polynomials of degree 2..12 (SplitMix64 seed 3), generated on device",
        "config": {"workload": f"uneven-gaussian-2^{args.log2n}: degree uniform 2..12, complex64 packed + u8 degree + "
                               f"i64 offsets, bin & pack + 12 persistent per-degree solvers, {W_PIX}x{H_PIX} histogram "
                               f"over [-3,3]x[-1.6875,1.6875]", "polys_per_gpu": n,
                   "coefficients": int(packed.numel()), "l2_flush": "inputs larger than L2 (0.94 GB per step)",
                   "parallelism": f"dp{world}",
                   "launch_shapes": {"per_degree": {str(d): {"block": int(tuning.block[d]),
                                                             "ctas_per_sm": int(tuning.ctas_per_sm[d]),
                                                             "lanes": int(tuning.lanes[d]),
                                                             "polish_warps": int(tuning.polish_warps[d])}
                                                    for d in range(2, 13)},
                                     "note": "each degree bin's fastest shape: warp-specialised (polish_warps > 0) "
                                             "where the tuner picked it and the bins have it (degrees <= 8), else "
                                             "its fastest one-role shape",
                                     "tuning_seconds": tuned["seconds"]}},
        "roofline": {"bound": "alu", "kernel": "whole step (pack + 12 uneven_solve_kernel launches)",
                     "achieved": (f32 + f64 * p32 / p64) / t / 1e12, "peak": p32 / 1e12, "unit": "TFLOP/s",
                     "frac": f32 / p32 / t + f64 / p64 / t, "traffic": None,
                     "fp32_frac": f32 / p32 / t, "fp64_frac": f64 / p64 / t, "peak_source": peak_src,
                     "note": "FP32-equivalent over the whole graph replay"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "status": {k: st[k] for k in ("status_ok", "status_not_converged", "status_rejected", "status_degenerate")},
        "sweeps_per_poly": st["sweeps"] / max(1, st["polys"]),
    }
    g32, g64 = algorithmic_flops(st_df)
    t_df = ms_df * 1e-3 / args.steps
    line["mixed_df_polish"] = {
        "value": n * world * args.steps / (ms_df * 1e-3), "unit": UNIT, "ms_per_step": ms_df / args.steps,
        "fp32_frac": g32 / p32 / t_df, "fp64_frac": g64 / p64 / t_df, "frac": g32 / p32 / t_df + g64 / p64 / t_df,
        "status": {k: st_df[k] for k in ("status_ok", "status_not_converged", "status_rejected",
                                         "status_degenerate")},
        "identical_image": bool(torch.equal(hist_df, hist)) if world == 1 else None,
        "note": "RD_POLISH_DF (Newton steps on the FP32 pipe, compensated Horner; FP64 final residual), one "
                "graph replay per step, each bin in the shape the tuner picked for this polish", "clocks": clk_df.summary()}
    if e2e is not None:
        line["e2e"] = e2e
    # the oracle's first chunk (polynomials 0..32767 of the stream), solved again
    # on the GPU with the timed launch shapes, for the root-error report
    sub = None
    if not args.no_cpu and n >= 32768:
        import numpy as np
        m = 32768
        off_h = off[:m + 1].cpu().numpy()
        ws_s = api.new_uneven_workspace(m, int(off_h[m]), torch.complex64, dev)
        r_s, st_s = api.roots_uneven(packed[:int(off_h[m])], deg[:m], off[:m + 1], ws_s, mode="mixed", params_=p,
                                     tuning=tuning)
        torch.cuda.synchronize()
        sub = (r_s.cpu().numpy(), st_s.cpu().numpy(), off_h)
    if not args.no_cpu:
        v, threads, done, first = cpu_oracle_rate_uneven(args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"first {done} polynomials of the same uneven stream, FP64 oracle solve + "
                                          f"histogram per degree, ~{args.cpu_seconds:.0f} s"}
        if sub is not None:
            r_g, st_g, off_g = sub
            per = {}
            for d, (sel, co_d, r_o, st_o) in first.items():
                base = off_g[sel] - sel  # where polynomial i's roots start in the packed roots
                g = r_g[base[:, None] + np.arange(d)[None, :]]
                per[d] = root_error_summary(g, st_g[sel], r_o, st_o, co_d, 1e-9, 1e3)
            line["root_error"] = {
                "subsample": "the first 32768 polynomials of the batch (the oracle's first chunk), GPU roots vs "
                             "the FP64 oracle (tol 1e-13) per degree, matched per polynomial; error "
                             "|z - z_oracle| / max(1, |z_oracle|), roots with kappa > 1e3 apart",
                "max_rel_err": max(e["max_rel_err"] for e in per.values()), "bar": 1e-9,
                "within_bar": all(e["within_bar"] for e in per.values()),
                "roots_compared": sum(e["roots_compared"] for e in per.values()),
                "ill_conditioned_roots": sum(e["ill_conditioned_roots"] for e in per.values()),
                "per_degree": {str(d): {k: e[k] for k in ("max_rel_err", "roots_compared", "ill_conditioned_roots",
                                                          "status_counts")} for d, e in sorted(per.items())}}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def _timed(step, args, dev, world, local_rank):
    """W warm-up steps, then K timed steps between CUDA events on the current
    stream (barrier + synchronize on both sides); returns (max-over-ranks ms
    for the K steps, clock summary, K). K is args.steps, raised when
    args.min_timed_s is set so that the timed region lasts at least that long
    (the clock sampler reads every 200 ms)."""
    import math

    import torch

    from paper_2507_02164_gb300 import dist as D
    for _ in range(args.warmup):
        step()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    steps = args.steps
    min_s = getattr(args, "min_timed_s", 0.0) or 0.0
    if min_s > 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        steps = max(steps, math.ceil(min_s * 1e3 / max(e0.elapsed_time(e1), 1e-3)))
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        t0.record(stream)
        for _ in range(steps):
            step()
        t1.record(stream)
        torch.cuda.synchronize()
    return D.max_over_ranks(t0.elapsed_time(t1), device=dev), clk.summary(), steps


PAPER_METRIC = "deg-6 complex polys rooted+binned/s with the paper's schedule (FP32, T=10 sweeps per root, Rayleigh shift)"


def run_paper(args, rank, world, local_rank):
    """The paper's own setting (Sec. IV: FP32, n = 6, T = 10, no convergence
    test) on the 2^26 Littlewood batch, fused with the histogram."""
    import torch

    from paper_2507_02164_gb300 import api, build, dist as D, workloads as WL
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = 1 << args.log2n
    start, _ = D.shard_range(n, rank)
    coeffs = WL.littlewood_soa_torch(SEED, start, n, dev)
    win = api.Window(*WINDOW)
    hist = api.new_hist(W_PIX, H_PIX, dev)
    stats = api.new_stats(dev)
    p = api.params("mixed", fixed_sweeps=10, shift="rayleigh", exc_period=0, polish_steps=0, polish_extra=0)

    def step():
        api.hist_clear(hist)
        api.hist_clear(stats)
        api.roots_density(coeffs, win, hist, mode="mixed", params_=p, stats=stats)

    ms, clk, steps = _timed(step, args, dev, world, local_rank)
    if rank != 0:
        return
    st = api.stats_dict(stats)
    value = n * world * steps / (ms * 1e-3)
    p32, p64, peak_src = roofline_peaks(torch, dev, local_rank)
    f32, f64 = algorithmic_flops(st)
    t = ms * 1e-3 / steps
    qr_per_s = value * st["sweeps"] / max(1, st["polys"])
    print(json.dumps({
        "metric": PAPER_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded Littlewood {1,-1,i,-i} degree-6 polynomials (SplitMix64 seed 2), generated on device",
        "config": {"workload": f"littlewood-deg6-2^{args.log2n}, fixed schedule T=10 (Alg. 2), Rayleigh shift, FP32 "
                               f"eigenvalues without polish, fused {W_PIX}x{H_PIX} histogram",
                   "l2_flush": "inputs larger than L2", "parallelism": f"dp{world}"},
        "roofline": {"bound": "alu", "kernel": "rd::solve_kernel<6, float, float2, MIXED> (fixed schedule)",
                     "achieved": (f32 + f64 * p32 / p64) / t / 1e12, "peak": p32 / 1e12, "unit": "TFLOP/s",
                     "frac": f32 / p32 / t + f64 / p64 / t, "traffic": None, "peak_source": peak_src},
        "gpu_launches": 3 * steps, "clocks": clk,
        "equiv_qr_decompositions_per_s": qr_per_s,
        "paper_context": {"fpga_qr_per_s": 16.5e6, "fpga_polys_per_s": 3.33e5, "rtx3060m_polys_per_s": 2.79e7,
                          "note": "paper's inputs unspecified; other hardware"},
    }), flush=True)


PIPELINE_METRIC = "sub-disks/s through L2 approximation + mixed roots + tile clip + histogram, f = sin(z^3) + 0.5 z"


def newton_move_of_kept(roots_w, centres, rho, tiles, nx, ny):
    """For every root w the tile clip keeps (z = c + rho w inside its own
    tile), one FP64 Newton step on f(z) = sin(z^3) + z/2 itself: its length is
    how far z lies from f's zero (the pipeline's accuracy check, bar 1e-6)."""
    import numpy as np
    w = roots_w.cpu().numpy().T
    c = centres.cpu().numpy()[:, None]
    z = c + rho * w
    with np.errstate(invalid="ignore"):
        tx = np.floor((z.real - tiles[0]) * nx / (tiles[1] - tiles[0]))
        ty = np.floor((tiles[3] - z.imag) * ny / (tiles[3] - tiles[2]))
    t = np.arange(c.shape[0])[:, None]
    kept = (tx == t % nx) & (ty == t // nx) & np.isfinite(z)
    zk = z[kept]
    f = np.sin(zk ** 3) + 0.5 * zk
    fp = 3 * zk ** 2 * np.cos(zk ** 3) + 0.5
    move = np.abs(f / fp)
    return {"kept_roots": int(kept.sum()), "max_newton_move": float(move.max(initial=0.0)),
            "bar": 1e-6, "within_bar": bool(move.max(initial=0.0) <= 1e-6)}


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s (MEASURED_PEAKS.json,
    written by the driver), else the fallback figure; and its source."""
    try:
        v = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "fallback (6.8 TB/s)"


def cpu_oracle_rate_pipeline(seconds: float):
    """The pipeline on the host cores for about `seconds`: f at the 16 x 32
    nodes of blocks of 4096 consecutive tiles of the 480 x 270 grid, oracle
    L2 fit, FP64 solve, map z = c + rho w, own-tile clip and histogram;
    returns (sub-disks/s, threads, sub-disks done)."""
    import numpy as np

    import oracle
    from paper_2507_02164_gb300 import workloads as WL
    oracle.build()
    win = (-4.0, 4.0, -2.25, 2.25)
    centres, rho, _, _ = WL.tiles(*win, 480, 270)
    nodes = oracle.l2_nodes(16, 32)
    block, done, elapsed, k, threads = 4096, 0, 0.0, 0, 0
    while elapsed < seconds:
        lo = (k * block) % centres.size
        idx = np.arange(lo, min(lo + block, centres.size))
        t0 = time.perf_counter()
        samples = WL.f_sin_cube(centres[idx][:, None] + rho * nodes[None, :])
        coeffs = oracle.l2_approx(samples)
        roots, _, _, threads = oracle.solve(coeffs)
        oracle.hist_tiled(oracle.affine(roots, centres[idx], rho), idx, 480, 270, win, W_PIX, H_PIX)
        elapsed += time.perf_counter() - t0
        done += idx.size
        k += 1
    return done / elapsed, threads, done


def run_pipeline(args, rank, world, local_rank, emit: bool = True):
    """The full pipeline: f(z) = sin(z^3) + 0.5 z on [-4,4]x[-2.25,2.25] in
    480 x 270 tiles; samples at the 16 x 32 nodes of every sub-disk are made
    on the device by torch outside the timed step; a step is L2
    approximation + fused mixed roots, tile clip and histogram. Beside it:
    the one-launch path (rd_field_density, f evaluated inside the kernel) and
    the split path's sampling time."""
    import torch

    from paper_2507_02164_gb300 import api, autotune, build, workloads as WL
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    win_t = (-4.0, 4.0, -2.25, 2.25)
    centres, rho, _, _ = WL.tiles(*win_t, 480, 270)
    c = torch.from_numpy(centres).to(dev)
    w = api.l2_sample_points(16, 32, dev)
    samples = WL.f_sin_cube(c[:, None] + rho * w[None, :]).contiguous()
    n = c.numel()
    coeffs = torch.empty((7, n), dtype=torch.complex128, device=dev)
    hist = api.new_hist(W_PIX, H_PIX, dev)
    stats = api.new_stats(dev)
    win = api.Window(*win_t)
    clip = api.make_clip(c, rho, 480, 270, win)
    # the roots step's launch shape, tuned at this batch size (complex128, degree 6)
    roots_shape = autotune.tune("mixed", dtype=torch.complex128, degrees=[6], n=n)["degrees"]["6"]
    p_roots = autotune.degree_params({"degrees": {"6": roots_shape}}, 6, "mixed")
    stream = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def make_step(precision):
        def step():
            api.hist_clear(hist)
            api.hist_clear(stats)
            e[0].record(stream)
            api.l2_approx(samples, 16, 32, 6, coeffs=coeffs, precision=precision)
            e[1].record(stream)
            api.roots_density(coeffs, win, hist, mode="mixed", params_=p_roots, clip=clip, stats=stats)
            e[2].record(stream)
        return step

    # the split path's producer: f at every node by torch (not in the timed
    # step; the evaluation above warmed torch's kernels)
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev_s[0].record(stream)
    samples = WL.f_sin_cube(c[:, None] + rho * w[None, :]).contiguous()
    ev_s[1].record(stream)
    torch.cuda.synchronize()
    sampling_ms = ev_s[0].elapsed_time(ev_s[1])

    # the one-launch path (rd_field_density): f, L2, roots, clip and histogram
    # in one kernel, no sample array
    spec = api.field_spec(win, 480, 270, radius=rho)
    e_f = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def fused_step():
        api.hist_clear(hist)
        api.hist_clear(stats)
        e_f[0].record(stream)
        api.field_density(spec, win, hist, mode="mixed", stats=stats)
        e_f[1].record(stream)

    ms_fused, clk_fused, k_fused = _timed(fused_step, args, dev, world, local_rank)
    fused_kernel_ms = e_f[0].elapsed_time(e_f[1])
    st_fused = api.stats_dict(stats)
    frames = render_frames(api, torch, dev, stream)

    # the FP64 L2 sums (RD_L2_FP64), for reference
    ms_fp64, _, k_fp64 = _timed(make_step("fp64"), args, dev, world, local_rank)
    l2_fp64_ms = e[0].elapsed_time(e[1])
    # the main leg: double-float L2 sums on the FP32 pipe (RD_L2_DF), same 1e-13 parity bar
    ms, clk, steps = _timed(make_step("df"), args, dev, world, local_rank)
    l2_ms = e[0].elapsed_time(e[1])
    solve_ms = e[1].elapsed_time(e[2])
    if rank != 0:
        return None
    st = api.stats_dict(stats)
    # accuracy (after the timed legs): every kept root of both paths, one FP64
    # Newton step on f itself; the step is the distance to f's zero there
    roots_t = torch.empty((6, n), dtype=torch.complex128, device=dev)
    hist_a = api.new_hist(W_PIX, H_PIX, dev)
    api.roots_density(coeffs, win, hist_a, mode="mixed", params_=p_roots, clip=clip, roots=roots_t)
    accuracy = {"split": newton_move_of_kept(roots_t, c, rho, win_t, 480, 270)}
    api.field_density(spec, win, hist_a, mode="mixed", roots=roots_t)
    accuracy["one_launch"] = newton_move_of_kept(roots_t, c, rho, win_t, 480, 270)
    p32, p64, peak_src = roofline_peaks(torch, dev, local_rank)
    # l2_approx algorithmic work per sub-disk: 512 samples x 16 B read, radial
    # sums 7 x 512 x 4 real flop (2 FMA), angular sums 7 x 32 x 8 flop
    l2_flops = n * (7 * 512 * 4 + 7 * 32 * 8)
    hbm, hbm_src = hbm_peak_gbs()
    f32r, f64r = algorithmic_flops(st)
    t_roots = solve_ms * 1e-3
    cpu = None
    if not args.no_cpu:
        v, threads, done = cpu_oracle_rate_pipeline(args.cpu_seconds)
        cpu = {"value": v, "unit": "sub-disks/s", "cores": threads, "kind": "oracle",
               "sample": f"{done} sub-disks (blocks of 4096 consecutive tiles): f at the nodes, FP64 oracle L2 fit, "
                         f"solve, map, own-tile clip and histogram, ~{args.cpu_seconds:.0f} s"}
    line = {
        "metric": PIPELINE_METRIC, "value": n * world * steps / (ms * 1e-3), "unit": "sub-disks/s",
        "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic: f(z) = sin(z^3) + 0.5 z sampled on the device at the quadrature nodes of every sub-disk",
        "config": {"workload": "480x270 tiles of 1/60 on [-4,4]x[-2.25,2.25], rho = tile half-diagonal, 16x32 polar "
                               "nodes, degree 6, mixed roots, clip to own tile, 1920x1080 histogram",
                   "sub_disks": n, "l2_flush": "inputs larger than L2 (1.06 GB of samples per step)",
                   "parallelism": f"dp{world}",
                   "roots_launch_shape": {x: roots_shape[x] for x in ("lanes", "block", "ctas_per_sm", "polish_warps",
                                                                      "ms")}},
        "l2_approx_ms": l2_ms, "roots_density_ms": solve_ms, "l2_precision": "double-float (RD_L2_DF)",
        "root_error": accuracy,
        "roofline": {"bound": "hbm", "kernel": "rd::l2_kernel_df<16, 6> (the step's larger kernel)",
                     "achieved": n * 512 * 16 / (l2_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": n * 512 * 16 / (l2_ms * 1e-3) / 1e9 / hbm, "traffic": None, "peak_source": hbm_src,
                     "note": "issue-bound double-float sums; bytes are the 1.06 GB of samples read once"},
        "roots_roofline": {"bound": "alu", "kernel": "rd_roots_density (mixed, clip)", "unit": "TFLOP/s",
                           "achieved": (f32r + f64r * p32 / p64) / t_roots / 1e12, "peak": p32 / 1e12,
                           "frac": f32r / p32 / t_roots + f64r / p64 / t_roots,
                           "fp32_frac": f32r / p32 / t_roots, "fp64_frac": f64r / p64 / t_roots,
                           "peak_source": peak_src},
        "l2_fp64": {"value": n * world * k_fp64 / (ms_fp64 * 1e-3), "ms_per_step": ms_fp64 / k_fp64,
                    "l2_approx_ms": l2_fp64_ms, "fp64_tflops": l2_flops / (l2_fp64_ms * 1e-3) / 1e12,
                    "fp64_frac": l2_flops / (l2_fp64_ms * 1e-3) / p64},
        "fused": {"value": n * world * k_fused / (ms_fused * 1e-3), "unit": "sub-disks/s",
                  "ms_per_step": ms_fused / k_fused, "field_kernel_ms": fused_kernel_ms,
                  "samples_per_s": n * 512 / (fused_kernel_ms * 1e-3), "kept_roots": st_fused["binned"],
                  "note": "rd_field_density: f evaluated in FP64 at the 16x32 nodes inside the kernel, L2, roots, "
                          "clip and histogram in one launch; no 1.06 GB sample array",
                  "clocks": clk_fused},
        "frames": frames,
        "split_end_to_end": {"sampling_ms": sampling_ms, "l2_plus_roots_ms": ms / steps,
                             "value": n / ((sampling_ms + ms / steps) * 1e-3),
                             "note": "torch evaluates f at every node into a 1.06 GB array, then the timed step"},
        "kept_roots": st["binned"], "clipped": st["clipped"],
        "status": {k: st[k] for k in ("status_ok", "status_not_converged", "status_rejected", "status_degenerate")},
        "gpu_launches": 4 * steps, "clocks": clk,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if emit:
        print(json.dumps(line), flush=True)
    return line


def small_batch_latency(api, WL, torch, dev, stream, reps=20, warmup=3):
    """Median latency of one roots + histogram call on 65,536 unit-disk
    degree-6 polynomials in plain FP64, replayed from a CUDA graph."""
    import numpy as np
    n = 65536
    co, true_roots = WL.unit_disk_roots(1, n)
    coeffs = torch.from_numpy(np.ascontiguousarray(co.T)).to(dev)
    hist = api.new_hist(W_PIX, H_PIX, dev)
    win = api.Window(-1.5, 1.5, -0.84375, 0.84375)
    # the launch shape tuned at this batch size (complex128, degree 6, plain)
    from paper_2507_02164_gb300 import autotune
    shape = autotune.tune("plain", dtype=torch.complex128, degrees=[6], n=n)["degrees"]["6"]
    p = autotune.degree_params({"degrees": {"6": shape}}, 6, "plain")
    api.roots_density(coeffs, win, hist, mode="plain", params_=p)  # loads the kernel, sizes the grid
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            api.hist_clear(hist)
            api.roots_density(coeffs, win, hist, mode="plain", params_=p)
    stream.wait_stream(side)
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    med = times[len(times) // 2]
    # root error of the same solve against the seeded roots the polynomials were built from
    r, st = api.roots_batched(coeffs, mode="plain", params_=p)
    err = root_error_summary(r.cpu().numpy().T, st.cpu().numpy(), true_roots, np.zeros(n, np.uint8), co, 1e-11, 1e2)
    err["reference"] = "the seeded roots each polynomial was expanded from (FP64)"
    return {"polys": n, "mode": "plain FP64 (tol 1e-13)", "median_ms": med, "min_ms": times[0],
            "polys_per_s": n / (med * 1e-3), "binned": int(hist.sum()), "root_error": err,
            "launch_shape": {k: shape[k] for k in ("lanes", "block", "ctas_per_sm", "ms")},
            "note": "unit-disk roots (seed 1), complex128, one graph replay = histogram clear + fused solve"}


def render_frames(api, torch, dev, stream, n_frames=60):
    """A zoom sequence of 1920x1080 root-density frames of sin(z^3) + z/2,
    each from 480x270 sub-disks with the one-launch path; frame f is copied
    to pinned host memory on a second stream while frame f+1 renders (two
    device and two host buffers): the headless counterpart of the paper's
    60 Hz display. Returns frames/s over the whole sequence, copies included."""
    import time
    copy_stream = torch.cuda.Stream(device=dev)
    hists = [api.new_hist(W_PIX, H_PIX, dev) for _ in range(2)]
    host = [torch.empty((H_PIX, W_PIX), dtype=torch.int32, pin_memory=True) for _ in range(2)]
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    target, zoom = complex(3.0, 0.0), 0.97  # towards the zeros near 2.87 +- 0.036i, 3.10 +- 0.035i

    def window(f):
        s = zoom ** f
        return api.Window(target.real - 4.0 * s, target.real + 4.0 * s, target.imag - 2.25 * s,
                          target.imag + 2.25 * s)

    def render(f):
        b = f % 2
        stream.wait_event(copied[b])  # the copy of frame f-2 out of this buffer is done
        api.hist_clear(hists[b])
        w = window(f)
        api.field_density(api.field_spec(w, 480, 270), w, hists[b], mode="mixed")
        rendered[b].record(stream)
        copy_stream.wait_event(rendered[b])
        with torch.cuda.stream(copy_stream):
            host[b].copy_(hists[b], non_blocking=True)
        copied[b].record(copy_stream)

    for f in range(3):
        render(f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for f in range(n_frames):
        render(f)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    return {"frames": n_frames, "fps": n_frames / sec, "ms_per_frame": 1e3 * sec / n_frames,
            "d2h_bytes_per_frame": W_PIX * H_PIX * 4, "sub_disks_per_frame": 480 * 270,
            "zoom": f"window 8 x 4.5 around {target}, scaled by {zoom} per frame",
            "last_frame_roots": int(host[(n_frames - 1) % 2].sum()),
            "note": "host wall clock over the sequence; frame f's copy to pinned memory overlaps frame f+1"}


ADJOINT_METRIC = "deg-6 polys/s through forward roots + implicit-differentiation adjoint"


def adjoint_flops(n: int, d: int = 6) -> float:
    """Algorithmic flops of the adjoint for n polynomials of degree d: per
    root, p'(z) by Horner (2d for k a_k, 8 (d-1) for the complex steps),
    u = conj(-1/p'(z)) grad_z (14), conj(z)^k for k <= d (6 d) and the d + 1
    accumulations grad_a_k += conj(z)^k u (8 (d + 1)): 24 d + 14 per root."""
    return float(n) * d * (24 * d + 14)


def cpu_oracle_rate_adjoint(seconds: float):
    """Oracle forward solve + implicit-differentiation adjoint of L = sum |z|^2
    on the adjoint workload's stream (complex-Gaussian, seed 4) for about
    `seconds`; returns (polys/s, threads, polys done)."""
    import numpy as np

    import oracle
    from paper_2507_02164_gb300 import workloads as WL
    oracle.build()
    chunk, done, elapsed, k, threads = 1 << 14, 0, 0.0, 0, 0
    while elapsed < seconds:
        co = WL.gaussian(4, np.arange(k * chunk, (k + 1) * chunk, dtype=np.uint64), 6)
        t0 = time.perf_counter()
        z, _, _, threads = oracle.solve(co)
        oracle.roots_backward(co, z, 2.0 * z)
        elapsed += time.perf_counter() - t0
        done += chunk
        k += 1
    return done / elapsed, threads, done


def run_adjoint(args, rank, world, local_rank, emit: bool = True):
    """2^20 complex-Gaussian degree-6 polynomials (seed 4): forward roots
    (mixed) and the adjoint for L = sum |z|^2 (grad_z = 2 z), timed
    separately, for complex128 and complex64 coefficients; and the whole
    soft-density loss step (roots, image, loss, pull-back, adjoint)."""
    import numpy as np
    import torch

    from paper_2507_02164_gb300 import api, autotune, build, workloads as WL
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_2507_02164_gb300 import splat as SP
    n = 1 << 20
    co = WL.gaussian(4, n, 6)
    out, shapes = {}, {}
    stream = torch.cuda.current_stream()
    # target image: the splat of a second seeded batch (2^16 polynomials)
    tgt_co = torch.from_numpy(np.ascontiguousarray(WL.gaussian(5, 1 << 16, 6).T)).to(dev)
    target = SP.splat(api.roots_batched(tgt_co, mode="mixed")[0])
    for name, dt in (("c128", torch.complex128), ("c64", torch.complex64)):
        coeffs = torch.from_numpy(np.ascontiguousarray(co.T)).to(dev).to(dt)
        # the forward solve in the autotuner's launch shape for this storage type
        shapes[name] = autotune.tune("mixed", dtype=dt, degrees=[6])["degrees"]["6"]
        p = autotune.degree_params({"degrees": {"6": shapes[name]}}, 6, "mixed")
        roots = torch.empty((6, n), dtype=torch.complex128, device=dev)
        status = torch.empty(n, dtype=torch.uint8, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

        def step():
            ev[0].record(stream)
            api.roots_batched(coeffs, mode="mixed", params_=p, roots=roots, status=status)
            ev[1].record(stream)
            api.roots_backward(coeffs, roots, 2.0 * roots)
            ev[2].record(stream)

        ms, clk, k = _timed(step, args, dev, world, local_rank)
        out[name] = {"ms_per_step": ms / k, "steps": k, "forward_ms": ev[0].elapsed_time(ev[1]),
                     "backward_ms": ev[1].elapsed_time(ev[2]), "value": n * world * k / (ms * 1e-3),
                     "clocks": clk}

        # the whole differentiation step through autograd: roots, soft-density
        # image, loss, the image's pull-back (CUDA splat kernels) and the adjoint
        co_g = coeffs.clone().requires_grad_(True)

        # complex64 coefficients carry ~1e-7: their image takes the FP32 stencil
        precision = "fp32" if name == "c64" else "fp64"

        def loss_step():
            co_g.grad = None
            z, _ = api.roots(co_g, "mixed", p)
            L = SP.loss(z, target, precision=precision)
            L.backward()

        ms_l, _, k_l = _timed(loss_step, args, dev, world, local_rank)
        out[name]["loss_step_ms"] = ms_l / k_l
        out[name]["loss_step_value"] = n * world * k_l / (ms_l * 1e-3)
        out[name]["splat_precision"] = precision
    if rank != 0:
        return None
    # roofline of the adjoint kernel: FP64 (complex128) / FP32 (complex64) flops
    p32, p64, peak_src = roofline_peaks(torch, dev, local_rank)
    for name, peak in (("c128", p64), ("c64", p32)):
        bw = out[name]["backward_ms"] * 1e-3
        out[name]["backward_roofline"] = {
            "bound": "alu", "kernel": f"rd::backward_kernel<6, {'double' if name == 'c128' else 'float'}>",
            "achieved": adjoint_flops(n) / bw / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": adjoint_flops(n) / bw / peak, "traffic": None, "peak_source": peak_src,
            "algorithmic_flops": adjoint_flops(n), "flops_per_poly": adjoint_flops(1)}
    # gradient parity on a sample: the GPU adjoint at the GPU roots vs the oracle's
    sample = np.arange(0, n, n // 4096, dtype=np.int64)[:4096]
    co_s = co[sample]
    cs = torch.from_numpy(np.ascontiguousarray(co_s.T)).to(dev)
    z_s, st_s = api.roots_batched(cs, mode="mixed")
    g_s = api.roots_backward(cs, z_s, 2.0 * z_s).cpu().numpy().T
    zz = z_s.cpu().numpy().T
    import oracle
    oracle.build()
    g_ref, _ = oracle.roots_backward(co_s, zz, 2.0 * zz)
    scale = np.maximum(np.abs(g_ref).max(axis=1, keepdims=True), 1e-300)
    grad_err = float((np.abs(g_s - g_ref) / scale).max())
    cpu = None
    if not args.no_cpu:
        v, threads, done = cpu_oracle_rate_adjoint(args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {done} polynomials of the same stream: FP64 oracle solve + adjoint of "
                         f"L = sum |z|^2, ~{args.cpu_seconds:.0f} s"}
    line = {
        "metric": ADJOINT_METRIC, "value": out["c128"]["value"], "unit": UNIT, "n_gpus": world,
        "steps": out["c128"]["steps"],
        "warmup": args.warmup, "ms_per_step": out["c128"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (c128) / f32 (c64)",
        "data": "synthetic: seeded complex-Gaussian degree-6 polynomials (SplitMix64 seed 4)",
        "config": {"workload": "2^20 deg-6, forward mixed roots + adjoint of L = sum |z|^2; loss_step: "
                               "L = sum |z|^2 + sum (D - T)^2 with D the 256x144 soft-density image "
                               "(sigma 1.5 px) of the roots, forward and backward through autograd",
                   "l2_flush": "none (inputs 112 MB c128, 56 MB c64)", "parallelism": f"dp{world}",
                   "launch_shapes": {k: {x: v[x] for x in ("lanes", "block", "ctas_per_sm", "polish_warps", "ms")}
                                     for k, v in shapes.items()}},
        "c128": out["c128"], "c64": out["c64"], "gpu_launches": 2 * out["c128"]["steps"],
        "clocks": out["c128"]["clocks"],
        "roofline": out["c128"]["backward_roofline"],
        "grad_error": {"sample": "4096 polynomials spread over the batch (complex128): GPU adjoint of L = sum |z|^2 "
                                 "at the GPU roots vs the oracle's adjoint at the same roots, relative to each "
                                 "polynomial's largest gradient", "max_rel_err": grad_err, "bar": 1e-12,
                       "within_bar": grad_err <= 1e-12},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if emit:
        print(json.dumps(line), flush=True)
    return line


def launch_plan(gpus: int, env, impl: str):
    """How `--gpus N` runs: ("run", world) in this process (N = 1, the
    reference arm, whose rank 0 alone works, or one rank of a launch whose
    WORLD_SIZE is N), ("exec", N) to start N ranks under
    torch.distributed.run, or ("error", message) when --gpus disagrees with
    the launcher's WORLD_SIZE."""
    if gpus < 1:
        return "error", "--gpus must be >= 1"
    ws = env.get("WORLD_SIZE")
    if ws is not None:
        world = int(ws)
        if world != gpus:
            return "error", f"--gpus {gpus} does not match WORLD_SIZE={world} of the launcher"
        return "run", world
    if gpus == 1 or impl == "reference":
        return "run", 1
    return "exec", gpus


def torchrun_argv(gpus: int, argv, port: int):
    """The command that starts `gpus` ranks of this script on one node (one
    process per GPU, rendezvous on 127.0.0.1)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
            "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *argv]


def _free_port() -> int:
    import socket
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def main():
    args = parse_args()
    if args.log2n is None:
        args.log2n = 26 if args.workload == "littlewood" else 24
    plan, val = launch_plan(args.gpus, os.environ, args.impl)
    if plan == "error":
        print(f"bench.py: {val}", file=sys.stderr)
        sys.exit(2)
    if plan == "exec":
        argv = torchrun_argv(val, sys.argv[1:], _free_port())
        os.execv(argv[0], argv)
    world = val
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        runner = {"uneven": run_uneven, "paper": run_paper, "pipeline": run_pipeline,
                  "adjoint": run_adjoint}.get(args.workload, run_ours)
        runner(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
