"""Launch-shape autotuner for the solve kernels.

For each degree the candidates are a threads-per-CTA size (64, 128, 256) and
a number of resident CTAs per SM (the occupancy maximum, or fewer). Each
candidate solves a probe batch of complex-Gaussian polynomials through the C
ABI (rd_roots_density, the fused path the benchmarks time) and is timed with
CUDA events; the fastest wins. The uneven-degree path takes one shape per
degree group (1-6, 7-9, 10-12): the candidate with the smallest summed time
over the group's degrees. Results are cached per GPU, mode and storage type in
a JSON file, so a process tunes once.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import api, workloads as WL

BLOCKS = (64, 128, 256)
GROUPS = ((1, 6), (7, 9), (10, 12))
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rootdensity_tuning.json")


def _occupancy_candidates(block: int):
    # 0 = the occupancy maximum the library computes; 1 and 2 trade
    # occupancy for fewer competing warps
    return (0, 1, 2) if block >= 128 else (0, 2, 4)


def _probe(degree: int, n: int, dtype, device):
    import numpy as np
    co = WL.gaussian(977 + degree, n, degree)
    return torch.from_numpy(np.ascontiguousarray(co.T)).to(device=device, dtype=dtype)


def time_shape(coeffs, mode: str, block: int, cps: int, reps: int = 3) -> float:
    """Median milliseconds of one fused solve + binning of `coeffs` with the given shape."""
    hist = api.new_hist(1920, 1080, coeffs.device)
    win = api.Window(-3.0, 3.0, -1.6875, 1.6875)
    p = api.params(mode, block=block, ctas_per_sm=cps)
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
    """{(block, cps): ms} for one degree, and the best shape."""
    coeffs = _probe(degree, n, dtype, device)
    res = {}
    for block in BLOCKS:
        for cps in _occupancy_candidates(block):
            try:
                res[(block, cps)] = time_shape(coeffs, mode, block, cps)
            except api.N.RootDensityError:
                continue  # shape not launchable (registers)
    best = min(res, key=res.get)
    return res, best


def choose_groups(tables: dict) -> list:
    """Per degree group, the shape with the least summed time over the group's
    tuned degrees among the shapes every one of them could launch; [0, 0]
    (library defaults) for a group without tuned degrees."""
    groups = []
    for lo, hi in GROUPS:
        ds = [d for d in tables if lo <= d <= hi]
        shapes = set.intersection(*(set(tables[d]) for d in ds)) if ds else set()
        if shapes:
            best = min(sorted(shapes), key=lambda sh: sum(tables[d][sh] for d in ds))
            groups.append([best[0], best[1]])
        else:
            groups.append([0, 0])
    return groups


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
    {"degrees": {d: {"block", "ctas_per_sm", "ms", "table"}}, "groups":
    [[block, cps] x 3], "seconds": time spent measuring}."""
    key = f"{_key(mode, dtype)}|n={n}"
    cache = load(cache_path) if cache_path else {}
    entry = cache.get(key, {}) if not force else {}
    t0 = time.perf_counter()
    for d in degrees:
        if str(d) in entry:
            continue
        res, best = tune_degree(d, mode, dtype, n)
        entry[str(d)] = {"block": best[0], "ctas_per_sm": best[1], "ms": res[best],
                         "table": [[b, c, t] for (b, c), t in sorted(res.items())]}
    spent = time.perf_counter() - t0
    if cache_path:
        cache[key] = entry
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    tables = {int(d): {(b, c): t for b, c, t in entry[str(d)]["table"]} for d in degrees}
    per_deg = {str(d): entry[str(d)] for d in degrees}
    return {"degrees": per_deg, "groups": choose_groups(tables), "seconds": spent, "probe_polys": n}


def uneven_tuning(result: dict):
    """rd_uneven_tuning from a tune() result."""
    g = result["groups"]
    return api.uneven_tuning(block=[x[0] for x in g], ctas_per_sm=[x[1] for x in g])


def degree_params(result: dict, degree: int, mode: str = "mixed"):
    """rd_params for a uniform batch of `degree` from a tune() result."""
    e = result["degrees"][str(degree)]
    return api.params(mode, block=e["block"], ctas_per_sm=e["ctas_per_sm"])
