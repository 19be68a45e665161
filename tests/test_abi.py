"""The C ABI library loads and exports every declared entry point; host-only
functions and argument validation need no GPU."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2507_02164_gb300 import _native as N
from paper_2507_02164_gb300 import build as B

HEADER = os.path.join(B.ROOT, "include", "rootdensity.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rd_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_loads():
    L = N.load()
    assert L.rd_abi_version() == N.ABI_VERSION == 2


def test_every_declared_symbol_is_exported_and_bound():
    L = N.load()
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
        assert name in N.SIGNATURES, f"{name} declared but not bound in _native.SIGNATURES"
    assert set(N.SIGNATURES) == set(names)


def test_struct_sizes_match_header_layout():
    assert ctypes.sizeof(N.TuneEntry) == 20 and ctypes.sizeof(N.Tuning) == 48
    assert ctypes.sizeof(N.Params) == 72
    assert ctypes.sizeof(N.Window) == 32
    assert ctypes.sizeof(N.Clip) == 64
    assert ctypes.sizeof(N.UnevenTuning) == 4 * 16 * 4
    assert ctypes.sizeof(N.FieldSpec) == 32 + 8 + 8 + 16 + 26 * 8
    assert N.STATS_WORDS == 15


def test_default_params():
    p = N.default_params(N.PLAIN_FP64)
    assert p.tol == 1e-13 and p.max_iters == 40 and p.shift == N.SHIFT_WILKINSON
    q = N.default_params(N.MIXED)
    assert q.tol == 4 * 2.0 ** -24 and q.polish_steps == 3 and q.collapse_tol == 1e-9
    assert q.polish_extra == 5 and q.fixed_sweeps == 0 and q.polish_mode == N.POLISH_FP64 and q.lanes == 0


@pytest.mark.parametrize("nr", [1, 2, 7, 16, 32])
def test_library_gauss_legendre_matches_numpy(nr):
    r = (ctypes.c_double * nr)()
    w = (ctypes.c_double * nr)()
    th = (ctypes.c_double * 32)()
    assert N.load().rd_l2_nodes(nr, 32, ctypes.cast(r, ctypes.c_void_p), ctypes.cast(th, ctypes.c_void_p),
                                ctypes.cast(w, ctypes.c_void_p)) == 0
    assert np.array_equal(np.array(th), 2.0 * np.pi * np.arange(32) / 32)
    t, wt = np.polynomial.legendre.leggauss(nr)
    assert np.allclose(np.array(r), 0.5 * (t + 1), atol=2e-16, rtol=0)
    assert np.allclose(np.array(w), 0.5 * wt, atol=0, rtol=1e-13)
    # exact for polynomials of degree < 2 nr: sum w_p r_p^k = 1/(k+1)
    rr, ww = np.array(r), np.array(w)
    for k in range(2 * nr):
        assert abs((ww * rr ** k).sum() - 1.0 / (k + 1)) <= 2e-15


def _err(rc):
    return rc, N.load().rd_last_error().decode()


def test_argument_validation_without_gpu():
    L = N.load()
    p = N.default_params(N.MIXED)
    null = ctypes.c_void_p(0)
    # degree outside 1..12
    rc, msg = _err(L.rd_roots_batched(null, N.C64, 13, 10, N.MIXED, ctypes.byref(p), null, null, null, null))
    assert rc == N.RD_EUNSUPPORTED and "degree" in msg
    # negative n
    rc, _ = _err(L.rd_roots_batched(null, N.C64, 6, -1, N.MIXED, ctypes.byref(p), null, null, null, null))
    assert rc == N.RD_EINVAL
    # null coefficients with work to do
    rc, msg = _err(L.rd_roots_batched(null, N.C64, 6, 5, N.MIXED, ctypes.byref(p), null, null, null, null))
    assert rc == N.RD_EINVAL and "coeffs" in msg
    # misaligned coefficient pointer (complex128 needs 16 bytes)
    rc, _ = _err(L.rd_roots_batched(ctypes.c_void_p(8), N.C128, 6, 5, N.MIXED, ctypes.byref(p), null, null,
                                    null, null))
    assert rc == N.RD_EINVAL
    # bad parameters
    bad = N.default_params(N.MIXED)
    bad.max_iters = 0
    rc, msg = _err(L.rd_roots_batched(ctypes.c_void_p(64), N.C64, 6, 5, N.MIXED, ctypes.byref(bad), null, null,
                                      null, null))
    assert rc == N.RD_EINVAL and "max_iters" in msg
    bad = N.default_params(N.MIXED)
    bad.block = 48
    rc, _ = _err(L.rd_roots_batched(ctypes.c_void_p(64), N.C64, 6, 5, N.MIXED, ctypes.byref(bad), null, null,
                                    null, null))
    assert rc == N.RD_EINVAL
    # empty batch is a no-op
    assert L.rd_roots_batched(null, N.C64, 6, 0, N.MIXED, ctypes.byref(p), null, null, null, null) == 0
    # density: inverted window, bad size, null hist
    h64 = ctypes.c_void_p(64)

    def dens(roots, status, n_roots, n_polys, win, Wd, Hd, clip, hist):
        return _err(L.rd_density_accumulate(roots, status, n_roots, n_polys, win, Wd, Hd, clip, hist, null, null))

    w_bad = N.Window(1.0, -1.0, -1.0, 1.0)
    assert dens(h64, null, 4, 0, w_bad, 16, 16, None, h64)[0] == N.RD_EINVAL
    w = N.Window(-1.0, 1.0, -1.0, 1.0)
    assert dens(h64, null, 4, 0, w, 0, 16, None, h64)[0] == N.RD_EINVAL
    assert dens(h64, null, 4, 0, w, 16, 16, None, null)[0] == N.RD_EINVAL
    nanw = N.Window(float("nan"), 1.0, -1.0, 1.0)
    assert dens(h64, null, 4, 0, nanw, 16, 16, None, h64)[0] == N.RD_EINVAL
    # the status mask and the clip need the roots grouped by polynomial
    rc, msg = dens(h64, h64, 4, 0, w, 16, 16, None, h64)
    assert rc == N.RD_EINVAL and "n_polys" in msg
    rc, msg = dens(h64, h64, 6, 4, w, 16, 16, None, h64)
    assert rc == N.RD_EINVAL and "multiple" in msg
    clip = N.Clip(centres=None, radius=0.1, tile_index=None, nx=4, ny=4, tiles=w)
    rc, msg = dens(h64, null, 8, 4, w, 16, 16, ctypes.byref(clip), h64)
    assert rc == N.RD_EINVAL and "centres" in msg
    clip = N.Clip(centres=64, radius=0.1, tile_index=None, nx=2, ny=1, tiles=w)
    rc, msg = dens(h64, null, 8, 4, w, 16, 16, ctypes.byref(clip), h64)
    assert rc == N.RD_EINVAL and "nx*ny" in msg
    assert dens(null, null, 0, 0, w, 16, 16, None, h64)[0] == 0  # nothing to bin
    # l2: nt must be 32, nr in 1..32
    def l2(s_, n, nr, nt, deg, prec, cen, rad, co, m):
        return _err(L.rd_l2_approx(s_, n, nr, nt, deg, prec, cen, rad, co, m, null))

    assert l2(h64, 4, 16, 16, 6, 0, null, 0.0, h64, None)[0] == N.RD_EUNSUPPORTED
    assert l2(h64, 4, 40, 32, 6, 0, null, 0.0, h64, None)[0] == N.RD_EINVAL
    assert l2(h64, 4, 16, 32, 6, 7, null, 0.0, h64, None)[0] == N.RD_EINVAL
    # the affine map: centres and radius are checked, then written into the clip
    m = N.Clip()
    assert l2(h64, 4, 16, 32, 6, 0, null, 0.5, h64, ctypes.byref(m))[0] == N.RD_EINVAL
    assert l2(h64, 4, 16, 32, 6, 0, h64, -1.0, h64, ctypes.byref(m))[0] == N.RD_EINVAL
    assert l2(null, 0, 16, 32, 6, 0, ctypes.c_void_p(4096), 0.25, null, ctypes.byref(m))[0] == 0
    assert m.centres == 4096 and m.radius == 0.25
    # l2 nodes: bad sizes
    buf = (ctypes.c_double * 64)()
    b = ctypes.cast(buf, ctypes.c_void_p)
    assert _err(L.rd_l2_nodes(16, 0, b, b, b))[0] == N.RD_EINVAL
    assert _err(L.rd_l2_nodes(33, 32, b, b, b))[0] == N.RD_EINVAL
    # uneven sizes beyond 2^32 polynomials or 2^40 coefficients
    assert L.rd_uneven_workspace_bytes(10, (1 << 40) + 1, N.C64) == 0
    assert L.rd_uneven_workspace_bytes(1 << 32, 10, N.C64) == 0
    assert L.rd_uneven_workspace_bytes(10, 100, 7) == 0
    rc, msg = _err(L.rd_roots_uneven(h64, N.C64, h64, h64, 10, (1 << 40) + 1, N.MIXED, None, None, None, 0, 0,
                                     null, null, null, null, h64, 1 << 20, null))
    assert rc == N.RD_EINVAL and "2^40" in msg
    rc, msg = _err(L.rd_roots_uneven_static(h64, N.C64, h64, h64, 10, (1 << 40) + 1, N.MIXED, None, None, None,
                                            0, 0, null, null, null, null, null))
    assert rc == N.RD_EINVAL
    # packed adjoint
    rc, _ = _err(L.rd_roots_backward_uneven(h64, 5, h64, h64, 4, 20, h64, h64, h64, null, null))
    assert rc == N.RD_EINVAL
    rc, msg = _err(L.rd_roots_backward_uneven(h64, N.C128, h64, h64, 4, (1 << 40) + 1, h64, h64, h64, null, null))
    assert rc == N.RD_EINVAL and "2^40" in msg
    rc, msg = _err(L.rd_roots_backward_uneven(h64, N.C128, null, h64, 4, 20, h64, h64, h64, null, null))
    assert rc == N.RD_EINVAL and "degrees" in msg
    assert L.rd_roots_backward_uneven(null, N.C128, null, null, 0, 0, null, null, null, null, null) == 0
    # autotuner and ALU probe: argument checks come before any device work
    t = N.Tuning()
    F = N.POLISH_FP64
    assert _err(L.rd_autotune(13, N.MIXED, F, N.C64, 1 << 16, 3, ctypes.byref(t), None, 0, None))[0] == \
        N.RD_EUNSUPPORTED
    assert _err(L.rd_autotune(6, N.MIXED, F, N.C64, 100, 3, ctypes.byref(t), None, 0, None))[0] == N.RD_EINVAL
    assert _err(L.rd_autotune(6, N.MIXED, F, N.C64, 1 << 16, 0, ctypes.byref(t), None, 0, None))[0] == N.RD_EINVAL
    assert _err(L.rd_autotune(6, N.MIXED, F, N.C64, 1 << 16, 3, None, None, 0, None))[0] == N.RD_EINVAL
    assert _err(L.rd_autotune(6, N.MIXED, 5, N.C64, 1 << 16, 3, ctypes.byref(t), None, 0, None))[0] == N.RD_EINVAL
    fl = ctypes.c_uint64()
    assert _err(L.rd_alu_peak(2, 10, 4, h64, ctypes.byref(fl), null))[0] == N.RD_EINVAL
    assert _err(L.rd_alu_peak(0, 0, 4, h64, ctypes.byref(fl), null))[0] == N.RD_EINVAL
    assert _err(L.rd_alu_peak(0, 10, 4, ctypes.c_void_p(65), ctypes.byref(fl), null))[0] == N.RD_EINVAL
    # backward: bad degree / null
    rc, _ = _err(L.rd_roots_backward(null, N.C128, 0, 4, null, null, null, null, null))
    assert rc == N.RD_EUNSUPPORTED
    rc, _ = _err(L.rd_roots_backward(null, N.C128, 6, 4, null, null, null, null, null))
    assert rc == N.RD_EINVAL
    assert L.rd_hist_clear(null, 0, null) == 0
    rc, _ = _err(L.rd_hist_clear(null, 5, null))
    assert rc == N.RD_EINVAL
    # lanes per polynomial: 0, 1 or 2; two lanes only with the FP64 polish
    bad = N.default_params(N.MIXED)
    bad.lanes = 3
    rc, msg = _err(L.rd_roots_batched(ctypes.c_void_p(64), N.C64, 6, 5, N.MIXED, ctypes.byref(bad), null, null,
                                      null, null))
    assert rc == N.RD_EINVAL and "lanes" in msg
    bad.lanes, bad.polish_mode = 2, N.POLISH_DF
    rc, msg = _err(L.rd_roots_batched(ctypes.c_void_p(64), N.C64, 6, 5, N.MIXED, ctypes.byref(bad), null, null,
                                      null, null))
    assert rc == N.RD_EINVAL and "lanes" in msg


def test_warp_specialised_argument_validation_without_gpu():
    """params.polish_warps / ring_slots: every bad combination is refused on
    the host before anything is launched."""
    L = N.load()
    null = ctypes.c_void_p(0)
    co = ctypes.c_void_p(64)

    def batched(degree=6, mode=N.MIXED, **kw):
        q = N.default_params(mode)
        for k, v in kw.items():
            setattr(q, k, v)
        return _err(L.rd_roots_batched(co, N.C64, degree, 5, mode, ctypes.byref(q), null, null, null, null))

    for kw, word in [(dict(polish_warps=16), "polish_warps"), (dict(polish_warps=-1), "polish_warps"),
                     (dict(polish_warps=2, ring_slots=1), "ring_slots"),
                     (dict(polish_warps=2, ring_slots=65), "ring_slots"),
                     (dict(polish_warps=2, block=544), "block"), (dict(block=512), "block"),
                     (dict(polish_warps=2, lanes=2), "polish_warps"),
                     (dict(polish_warps=4, block=128), "polish_warps"),  # no sweep warp left
                     (dict(polish_warps=1, block=512), "block")]:  # degree 8: at most 256 threads
        rc, msg = batched(8 if kw.get("block") == 512 else 6, **kw)
        assert rc == N.RD_EINVAL and word in msg, (kw, rc, msg)
    rc, msg = batched(mode=N.PLAIN_FP64, polish_warps=2)
    assert rc == N.RD_EINVAL and "polish_warps" in msg
    # uneven batches and the one-launch field path have no warp-specialised form
    q = N.default_params(N.MIXED)
    q.polish_warps = 2
    rc, msg = _err(L.rd_roots_uneven(co, N.C64, null, null, 0, 0, N.MIXED, ctypes.byref(q), None, None, 0, 0, null,
                                     null, null, null, null, 0, null))
    assert rc == N.RD_EINVAL and "polish_warps" in msg
    # the bounded-wait self-test: 1 <= n <= 1024, status and stats required
    for n, st, stats in [(0, co, co), (1025, co, co), (32, null, co), (32, co, null)]:
        rc, _ = _err(L.rd_ws_selftest_timeout(co, n, st, stats, null))
        assert rc == N.RD_EINVAL


def test_field_density_argument_validation_without_gpu():
    L = N.load()
    null = ctypes.c_void_p(0)
    p = N.default_params(N.MIXED)
    w = N.Window(-1.0, 1.0, -1.0, 1.0)

    def spec(**kw):
        s = N.FieldSpec()
        s.tiles = N.Window(-1.0, 1.0, -1.0, 1.0)
        s.nx, s.ny, s.nr, s.degree = 8, 8, 16, 6
        for k, v in kw.items():
            setattr(s, k, v)
        return s

    def call(f, sp, params=p, hist=ctypes.c_void_p(64)):
        return _err(L.rd_field_density(f, ctypes.byref(sp) if sp is not None else None, N.MIXED,
                                       ctypes.byref(params), w, 16, 16, hist, null, null, null, null, null))

    rc, msg = call(7, spec())
    assert rc == N.RD_EINVAL and "RD_F_" in msg
    rc, msg = call(N.F_SIN_CUBE, None)
    assert rc == N.RD_EINVAL and "spec" in msg
    rc, msg = call(N.F_SIN_CUBE, spec(nx=0))
    assert rc == N.RD_EINVAL and "nx" in msg
    rc, msg = call(N.F_SIN_CUBE, spec(tiles=N.Window(1.0, -1.0, -1.0, 1.0)))
    assert rc == N.RD_EINVAL and "tiles" in msg
    rc, msg = call(N.F_SIN_CUBE, spec(nr=8))
    assert rc == N.RD_EUNSUPPORTED and "nr" in msg
    rc, msg = call(N.F_SIN_CUBE, spec(degree=4))
    assert rc == N.RD_EUNSUPPORTED and "degree" in msg
    rc, msg = call(N.F_POLY, spec(poly_degree=13))
    assert rc == N.RD_EINVAL and "poly_degree" in msg
    sp = spec(poly_degree=2)
    sp.poly[3] = float("inf")
    rc, msg = call(N.F_POLY, sp)
    assert rc == N.RD_EINVAL and "poly" in msg
    rc, msg = call(N.F_SIN_CUBE, spec(), hist=null)
    assert rc == N.RD_EINVAL and "hist" in msg
    two = N.default_params(N.MIXED)
    two.lanes = 2
    rc, msg = call(N.F_SIN_CUBE, spec(), params=two)
    assert rc == N.RD_EINVAL and "lanes" in msg


def test_python_binding_raises_on_error():
    with pytest.raises(N.RootDensityError):
        N.call("rd_hist_clear", ctypes.c_void_p(0), 5, ctypes.c_void_p(0))


def test_device_accessibility_query_without_gpu():
    """No GPU: nothing is device-accessible, and the query does not fail."""
    L = N.load()
    buf = (ctypes.c_char * 64)()
    assert L.rd_pointer_is_device_accessible(ctypes.cast(buf, ctypes.c_void_p)) == 0
    assert L.rd_pointer_is_device_accessible(None) == 0


def test_host_inputs_must_be_mapped_page_locked_memory():
    import torch
    from paper_2507_02164_gb300 import api
    with pytest.raises(ValueError, match="page-locked"):
        api.roots_batched(torch.zeros((7, 4), dtype=torch.complex64), mode="mixed")
