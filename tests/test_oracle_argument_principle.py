"""Pin of the oracle's full pipeline (tiles -> L2 fit -> roots -> own-tile
clip) against the argument principle, which counts the zeros of f inside a
tile without any polynomial fit: (1 / 2 pi) times the change of arg f along
the tile's boundary, sampled adaptively in FP64. For f(z) = sin(z^3) + z/2 on
the 480 x 270 tiles of [-4,4] x [-2.25,2.25], every tile that keeps a root
and 400 seeded random tiles: the number of roots the pipeline keeps in a
tile equals its winding number, except tiles whose boundary passes through a
zero (their winding number is not an integer: the real zeros lie on the row
edge y = 0, and z = 0 is a corner)."""
from __future__ import annotations

import math

import numpy as np

from paper_2507_02164_gb300 import workloads as WL

WIN = (-4.0, 4.0, -2.25, 2.25)
NX, NY = 480, 270


def _edge_arg(a: complex, b: complex, n: int = 32, depth: int = 14):
    """Change of arg f along the segment a -> b, refining any step whose arg
    change exceeds pi/4 (so the unwrapping cannot skip a turn); also the
    smallest and largest |f| seen (a zero on the segment draws the refined
    samples onto it)."""
    z = a + (b - a) * np.linspace(0.0, 1.0, n + 1)
    v = WL.f_sin_cube(z)
    with np.errstate(divide="ignore", invalid="ignore"):  # f = 0 exactly at z = 0 (a tile corner)
        d = np.angle(v[1:] / v[:-1])
    total, lo, hi = 0.0, float(np.abs(v).min()), float(np.abs(v).max())
    for i in range(n):
        if abs(d[i]) > math.pi / 4 and depth > 0:
            t, l, h = _edge_arg(z[i], z[i + 1], 8, depth - 1)
            total, lo, hi = total + t, min(lo, l), max(hi, h)
        else:
            total += float(d[i])
    return total, lo, hi


def _winding(t: int):
    """(winding number of f along tile t's boundary, min |f| / max |f| on it)."""
    iy, ix = divmod(t, NX)
    w = (WIN[1] - WIN[0]) / NX
    h = (WIN[3] - WIN[2]) / NY
    x0, y1 = WIN[0] + ix * w, WIN[3] - iy * h
    c = [complex(x0, y1 - h), complex(x0 + w, y1 - h), complex(x0 + w, y1), complex(x0, y1)]  # counter-clockwise
    parts = [_edge_arg(c[k], c[(k + 1) % 4]) for k in range(4)]
    return sum(p[0] for p in parts) / (2 * math.pi), min(p[1] for p in parts) / max(p[2] for p in parts)


def test_kept_roots_per_tile_equal_the_winding_number(orc):
    centres, rho, _, _ = WL.tiles(*WIN, NX, NY)
    nodes = orc.l2_nodes(16, 32)
    kept = np.zeros(centres.size, np.int64)
    for c0 in range(0, centres.size, 16200):
        c = centres[c0:c0 + 16200]
        co = orc.l2_approx(WL.f_sin_cube(c[:, None] + rho * nodes[None, :]))
        r, _, _, _ = orc.solve(co)
        z = orc.affine(r, c, rho)
        t = np.arange(c0, c0 + c.size)[:, None]
        with np.errstate(invalid="ignore"):
            tx = np.floor((z.real - WIN[0]) * NX / (WIN[1] - WIN[0]))
            ty = np.floor((WIN[3] - z.imag) * NY / (WIN[3] - WIN[2]))
        kept[c0:c0 + c.size] = ((tx == t % NX) & (ty == t // NX) & np.isfinite(z)).sum(axis=1)
    with_roots = np.nonzero(kept)[0]
    assert 55 <= with_roots.size <= 70
    rand = np.random.default_rng(20).choice(centres.size, 400, replace=False)
    checked = excluded = zero_free = 0
    for t in np.unique(np.concatenate([with_roots, rand])):
        wnd, floor_ratio = _winding(int(t))
        if floor_ratio < 1e-8 or abs(wnd - round(wnd)) > 0.05:  # the boundary passes through a zero
            excluded += 1
            continue
        assert kept[t] == round(wnd), (int(t), int(kept[t]), wnd)
        checked += 1
        zero_free += round(wnd) == 0
    assert checked >= 400 and excluded <= 12 and checked - zero_free >= 45, (checked, excluded, zero_free)
