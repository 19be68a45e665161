"""Launch-shape autotuner: a per-process cache over the library's rd_autotune.

rd_autotune (C ABI, csrc/rd_tune.cu) times every candidate launch shape of the
fused solve for one degree, mode and storage type on a probe batch of
complex-Gaussian polynomials: lanes per polynomial (1, or 2 sharing a matrix),
threads per CTA, resident CTAs per SM, and for the mixed mode the
warp-specialised CTAs (params.polish_warps: some warps polish what the others
sweep). The fastest shape serves uniform batches; the fastest shape without
warp specialisation serves the uneven-degree bins, whose per-degree kernels
have no warp-specialised form. This module calls it once per degree and
caches the results in a JSON file keyed by GPU, mode, storage type, probe
size and a hash of the library's sources, so that a process tunes once and a
rebuilt library is tuned again.
"""
from __future__ import annotations

import ctypes
import json
import os
import time

import torch

from . import _native as N
from . import api, build

CACHE_FORMAT = 5  # table rows [lanes, block, ctas_per_sm, polish_warps, ms]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rootdensity_tuning.json")
TABLE_CAP = 64


def _entry(e) -> tuple:
    return (int(e.lanes), int(e.block), int(e.ctas_per_sm), int(e.polish_warps))


POLISH = {"fp64": N.POLISH_FP64, "df": N.POLISH_DF}


def tune_degree(degree: int, mode: str = "mixed", dtype=torch.complex64, n: int = 1 << 18, reps: int = 3,
                polish: str = "fp64"):
    """One rd_autotune call: ({(lanes, block, cps, polish_warps): ms}, the best
    shape, the best shape with polish_warps = 0). ms < 0: not launchable.
    polish: "fp64" or "df" (the mixed mode's polish, rd_polish)."""
    t = N.Tuning()
    table = (N.TuneEntry * TABLE_CAP)()
    used = ctypes.c_int(0)
    N.call("rd_autotune", degree, api._mode(mode), POLISH[polish], api.DTYPES[dtype], n, reps, ctypes.byref(t), table,
           TABLE_CAP, ctypes.byref(used))
    res = {_entry(e): float(e.ms) for e in table[:used.value]}
    return res, (_entry(t.best), float(t.best.ms)), (_entry(t.one_role), float(t.one_role.ms))


def cache_key(mode: str, dtype, n: int, polish: str = "fp64") -> str:
    name = torch.cuda.get_device_name()
    kind = "c64" if dtype == torch.complex64 else "c128"
    m = f"{mode}-{polish}" if mode == "mixed" else mode
    return f"{name}|{m}|{kind}|n={n}|lib={build.source_hash()}|v{CACHE_FORMAT}"


def load(cache_path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(cache_path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(mode: str = "mixed", dtype=torch.complex64, degrees=range(1, 13), n: int = 1 << 20,
         cache_path: str | None = DEFAULT_CACHE, force: bool = False, polish: str = "fp64") -> dict:
    """Tune every requested degree; degrees already in the cache (same GPU,
    mode and polish, storage type, probe size and library sources) are not
    re-measured.
    Returns {"degrees": {d: {"lanes", "block", "ctas_per_sm", "polish_warps",
    "ms", "one_role": {"lanes", "block", "ctas_per_sm", "ms"}, "table"}},
    "seconds": time spent measuring, "probe_polys": n}."""
    key = cache_key(mode, dtype, n, polish)
    cache = load(cache_path) if cache_path else {}
    entry = cache.get(key, {}) if not force else {}
    t0 = time.perf_counter()
    for d in degrees:
        if str(d) in entry:
            continue
        res, (best, ms), (one, one_ms) = tune_degree(d, mode, dtype, n, polish=polish)
        entry[str(d)] = {"lanes": best[0], "block": best[1], "ctas_per_sm": best[2], "polish_warps": best[3],
                         "ms": ms,
                         "one_role": {"lanes": one[0], "block": one[1], "ctas_per_sm": one[2], "ms": one_ms},
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


UNEVEN_WS_MAX_DEG = 8  # the uneven bins have a warp-specialised form up to this degree


def uneven_tuning(result: dict):
    """rd_uneven_tuning (per degree) from a tune() result: each degree's
    fastest shape where the bins have it (the warp-specialised form up to
    degree 8), else its fastest one-role shape."""
    deg = {}
    for d, e in result["degrees"].items():
        if int(d) <= UNEVEN_WS_MAX_DEG and e.get("polish_warps", 0) > 0:
            deg[d] = {"block": e["block"], "ctas_per_sm": 0, "lanes": 1, "polish_warps": e["polish_warps"]}
        else:
            o = e.get("one_role", e)
            deg[d] = {"block": o["block"], "ctas_per_sm": o["ctas_per_sm"], "lanes": o["lanes"], "polish_warps": 0}
    return api.uneven_tuning(block={int(d): e["block"] for d, e in deg.items()},
                             ctas_per_sm={int(d): e["ctas_per_sm"] for d, e in deg.items()},
                             lanes={int(d): e["lanes"] for d, e in deg.items()},
                             polish_warps={int(d): e["polish_warps"] for d, e in deg.items()})


def degree_params(result: dict, degree: int, mode: str = "mixed", polish: str = "fp64"):
    """rd_params for a uniform batch of `degree` from a tune() result (made
    with the same polish)."""
    e = result["degrees"][str(degree)]
    extra = {"polish_mode": POLISH[polish]} if mode == "mixed" else {}
    return api.params(mode, block=e["block"], ctas_per_sm=e["ctas_per_sm"], lanes=e["lanes"],
                      polish_warps=e.get("polish_warps", 0), **extra)
