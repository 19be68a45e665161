"""Launch-shape autotuner for the solve kernels.

For each degree the candidates are the lanes per polynomial (one thread per
matrix, or two lanes sharing it; degree >= 2), a threads-per-CTA size (32,
64, 128, 256; small CTAs spread a small batch over more SMs) and a number of resident CTAs per SM (the occupancy maximum, or
fewer), all with every warp sweeping and then polishing its own polynomials;
and, for the mixed mode, warp-specialised CTAs (params.polish_warps: some
warps polish what the others sweep) of several sizes and splits. Each
candidate solves a probe batch of complex-Gaussian polynomials through the C
ABI (rd_roots_density, the fused path the benchmarks time) and is timed with
CUDA events; the fastest wins for uniform batches. The uneven-degree path
launches one kernel per degree bin, which has no warp-specialised form, and
takes each degree's fastest one-role shape. Results are cached per GPU, mode
and storage type in a JSON file, so a process tunes once.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import api, workloads as WL

BLOCKS = (32, 64, 128, 256)
CACHE_FORMAT = 4  # table rows [lanes, block, ctas_per_sm, polish_warps, ms]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rootdensity_tuning.json")


def _occupancy_candidates(block: int):
    # 0 = the occupancy maximum the library computes; 1 and 2 trade
    # occupancy for fewer competing warps
    return (0, 1, 2) if block >= 128 else (0, 2, 4)


def _probe(degree: int, n: int, dtype, device):
    import numpy as np
    co = WL.gaussian(977 + degree, n, degree)
    return torch.from_numpy(np.ascontiguousarray(co.T)).to(device=device, dtype=dtype)


def lane_candidates(degree: int):
    return (1, 2) if degree >= 2 else (1,)


def ws_candidates(degree: int):
    """(block, polish_warps) of the warp-specialised shapes: up to 16 warps per
    CTA at degree <= 6 (128 registers), up to 8 above (255 registers). One
    polish warp keeps about one FP64 instruction in flight, so the FP64 pipe
    wants about ten of them per SM."""
    if degree <= 6:
        return ((512, 8), (512, 9), (512, 10), (512, 11), (256, 4), (256, 5), (192, 3), (192, 4))
    return ((96, 1), (96, 2), (128, 1), (128, 2), (192, 2), (192, 3), (192, 4), (256, 3), (256, 4))


def time_shape(coeffs, mode: str, block: int, cps: int, reps: int = 3, lanes: int = 1,
               polish_warps: int = 0) -> float:
    """Median milliseconds of one fused solve + binning of `coeffs` with the given shape."""
    hist = api.new_hist(1920, 1080, coeffs.device)
    win = api.Window(-3.0, 3.0, -1.6875, 1.6875)
    p = api.params(mode, block=block, ctas_per_sm=cps, lanes=lanes, polish_warps=polish_warps)
    api.roots_density(coeffs, win, hist, mode=mode, params_=p)  # warm-up (and launch check)
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        api.roots_density(coeffs, win, hist, mode=mode, params_=p)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def tune_degree(degree: int, mode: str = "mixed", dtype=torch.complex64, n: int = 1 << 18, device="cuda"):
    """{(lanes, block, cps, polish_warps): ms} for one degree, the best shape,
    and the best one-role shape (polish_warps 0)."""
    coeffs = _probe(degree, n, dtype, device)
    res = {}
    for lanes in lane_candidates(degree):
        for block in BLOCKS:
            for cps in _occupancy_candidates(block):
                try:
                    res[(lanes, block, cps, 0)] = time_shape(coeffs, mode, block, cps, lanes=lanes)
                except api.N.RootDensityError:
                    continue  # shape not launchable (registers)
    if mode == "mixed":
        for block, pw in ws_candidates(degree):
            res[(1, block, 0, pw)] = time_shape(coeffs, mode, block, 0, polish_warps=pw)
    return res, best_shape(res), best_shape({k: v for k, v in res.items() if k[3] == 0})


def best_shape(table: dict):
    """The fastest shape of a table; ties go to the smaller tuple."""
    return min(sorted(table), key=lambda sh: table[sh])


def _key(mode: str, dtype) -> str:
    name = torch.cuda.get_device_name()
    return f"{name}|{mode}|{'c64' if dtype == torch.complex64 else 'c128'}"


def load(cache_path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(cache_path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(mode: str = "mixed", dtype=torch.complex64, degrees=range(1, 13), n: int = 1 << 20,
         cache_path: str | None = DEFAULT_CACHE, force: bool = False) -> dict:
    """Tune every requested degree; degrees already in the cache (same GPU,
    mode, storage type and probe size) are not re-measured. Returns
    {"degrees": {d: {"lanes", "block", "ctas_per_sm", "polish_warps", "ms",
    "one_role": {"lanes", "block", "ctas_per_sm", "ms"}, "table"}},
    "seconds": time spent measuring, "probe_polys": n}."""
    key = f"{_key(mode, dtype)}|n={n}|v{CACHE_FORMAT}"
    cache = load(cache_path) if cache_path else {}
    entry = cache.get(key, {}) if not force else {}
    t0 = time.perf_counter()
    for d in degrees:
        if str(d) in entry:
            continue
        res, best, one = tune_degree(d, mode, dtype, n)
        entry[str(d)] = {"lanes": best[0], "block": best[1], "ctas_per_sm": best[2], "polish_warps": best[3],
                         "ms": res[best],
                         "one_role": {"lanes": one[0], "block": one[1], "ctas_per_sm": one[2], "ms": res[one]},
                         "table": [[la, b, c, pw, t] for (la, b, c, pw), t in sorted(res.items())]}
    spent = time.perf_counter() - t0
    if cache_path:
        cache[key] = entry
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    per_deg = {str(d): entry[str(d)] for d in degrees}
    return {"degrees": per_deg, "seconds": spent, "probe_polys": n}


def uneven_tuning(result: dict):
    """rd_uneven_tuning (per degree) from a tune() result: each degree's
    fastest one-role shape (the uneven bins have no warp-specialised form)."""
    deg = {d: e.get("one_role", e) for d, e in result["degrees"].items()}
    return api.uneven_tuning(block={int(d): e["block"] for d, e in deg.items()},
                             ctas_per_sm={int(d): e["ctas_per_sm"] for d, e in deg.items()},
                             lanes={int(d): e["lanes"] for d, e in deg.items()})


def degree_params(result: dict, degree: int, mode: str = "mixed"):
    """rd_params for a uniform batch of `degree` from a tune() result."""
    e = result["degrees"][str(degree)]
    return api.params(mode, block=e["block"], ctas_per_sm=e["ctas_per_sm"], lanes=e["lanes"],
                      polish_warps=e.get("polish_warps", 0))
