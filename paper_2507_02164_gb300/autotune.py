"""Launch-shape autotuner for the solve kernels.

For each degree the candidates are the lanes per polynomial (one thread per
matrix, or two lanes sharing it; degree >= 2), a threads-per-CTA size (64,
128, 256) and a number of resident CTAs per SM (the occupancy maximum, or
fewer). Each candidate solves a probe batch of complex-Gaussian polynomials
through the C ABI (rd_roots_density, the fused path the benchmarks time) and
is timed with CUDA events; the fastest wins. The uneven-degree path launches
one kernel per degree bin and takes each degree's own winner. Results are
cached per GPU, mode and storage type in a JSON file, so a process tunes once.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import api, workloads as WL

BLOCKS = (64, 128, 256)
CACHE_FORMAT = 2  # table rows [lanes, block, ctas_per_sm, ms]
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


def time_shape(coeffs, mode: str, block: int, cps: int, reps: int = 3, lanes: int = 1) -> float:
    """Median milliseconds of one fused solve + binning of `coeffs` with the given shape."""
    hist = api.new_hist(1920, 1080, coeffs.device)
    win = api.Window(-3.0, 3.0, -1.6875, 1.6875)
    p = api.params(mode, block=block, ctas_per_sm=cps, lanes=lanes)
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
    """{(lanes, block, cps): ms} for one degree, and the best shape."""
    coeffs = _probe(degree, n, dtype, device)
    res = {}
    for lanes in lane_candidates(degree):
        for block in BLOCKS:
            for cps in _occupancy_candidates(block):
                try:
                    res[(lanes, block, cps)] = time_shape(coeffs, mode, block, cps, lanes=lanes)
                except api.N.RootDensityError:
                    continue  # shape not launchable (registers)
    return res, best_shape(res)


def best_shape(table: dict):
    """The fastest (lanes, block, cps) of a table; ties go to the smaller tuple."""
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
    {"degrees": {d: {"lanes", "block", "ctas_per_sm", "ms", "table"}},
    "seconds": time spent measuring, "probe_polys": n}."""
    key = f"{_key(mode, dtype)}|n={n}|v{CACHE_FORMAT}"
    cache = load(cache_path) if cache_path else {}
    entry = cache.get(key, {}) if not force else {}
    t0 = time.perf_counter()
    for d in degrees:
        if str(d) in entry:
            continue
        res, best = tune_degree(d, mode, dtype, n)
        entry[str(d)] = {"lanes": best[0], "block": best[1], "ctas_per_sm": best[2], "ms": res[best],
                         "table": [[la, b, c, t] for (la, b, c), t in sorted(res.items())]}
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
    """rd_uneven_tuning (per degree) from a tune() result."""
    deg = result["degrees"]
    return api.uneven_tuning(block={int(d): e["block"] for d, e in deg.items()},
                             ctas_per_sm={int(d): e["ctas_per_sm"] for d, e in deg.items()},
                             lanes={int(d): e["lanes"] for d, e in deg.items()})


def degree_params(result: dict, degree: int, mode: str = "mixed"):
    """rd_params for a uniform batch of `degree` from a tune() result."""
    e = result["degrees"][str(degree)]
    return api.params(mode, block=e["block"], ctas_per_sm=e["ctas_per_sm"], lanes=e["lanes"])
