"""GPU tests of the warp-specialised RD_MIXED solver (params.polish_warps > 0):
sweep warps hand FP32 eigenvalues to polish warps through a shared-memory
ring. The polish, check, store and binning are the one-role kernel's own
code, so roots, status, histogram and counters must equal that kernel's bit
for bit, for every degree, storage type, launch shape and ragged batch size;
one case also goes to the oracle directly. The bounded waits are exercised by
the self-test entry point, which starves the polish warps on purpose."""
from __future__ import annotations

import time

import numpy as np
import pytest
import torch

from paper_2507_02164_gb300 import api, workloads as WL
from tests.gpu_common import check_rejected, compare_roots, require_gpu, to_soa

pytestmark = pytest.mark.gpu

W, H = 1920, 1080
WIN2 = api.Window(-2.0, 2.0, -1.125, 1.125)
WIN3 = api.Window(-3.0, 3.0, -1.6875, 1.6875)


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _run(coeffs, degree, win, **kw):
    n = coeffs.shape[1]
    p = api.params("mixed", **kw)
    hist = api.new_hist(W, H, coeffs.device)
    stats = api.new_stats(coeffs.device)
    roots = torch.empty((degree, n), dtype=torch.complex128, device=coeffs.device)
    status = torch.empty(n, dtype=torch.uint8, device=coeffs.device)
    api.roots_density(coeffs, win, hist, "mixed", p, roots=roots, status=status, stats=stats)
    torch.cuda.synchronize()
    return roots, status, hist, api.stats_dict(stats)


def _same(a, b):
    ra, sa, ha, ta = a
    rb, sb, hb, tb = b
    assert torch.equal(torch.view_as_real(ra).view(torch.int64), torch.view_as_real(rb).view(torch.int64))
    assert torch.equal(sa, sb)
    assert torch.equal(ha, hb)
    assert ta == tb, {k: (ta[k], tb[k]) for k in ta if ta[k] != tb[k]}
    assert ta["wait_timeouts"] == 0


# (block, polish_warps, ring_slots): one and two CTAs per SM, minimal rings,
# one sweep warp per CTA, more polish than sweep warps
SHAPES_LOW = [(512, 4, 0), (512, 8, 16), (256, 2, 2), (64, 1, 2), (96, 2, 3), (512, 1, 64)]
SHAPES_HIGH = [(256, 2, 0), (256, 6, 5), (128, 1, 2)]


@pytest.mark.parametrize("n", [1, 31, 33, 4097, 100003])
@pytest.mark.parametrize("shape", SHAPES_LOW)
def test_littlewood_bit_identical_to_one_role_kernel(dev, n, shape):
    block, pw, slots = shape
    co = WL.littlewood_soa_torch(2, 12345, n, dev)
    ref = _run(co, 6, WIN2)
    got = _run(co, 6, WIN2, block=block, polish_warps=pw, ring_slots=slots)
    _same(got, ref)


@pytest.mark.parametrize("degree", list(range(1, 13)))
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_every_degree_bit_identical(dev, degree, dtype):
    n = 3000 + 17 * degree
    co = to_soa(WL.gaussian(200 + degree, n, degree), dev, dtype)
    ref = _run(co, degree, WIN3)
    shapes = SHAPES_LOW[:3] if degree <= 6 else SHAPES_HIGH
    for block, pw, slots in shapes:
        _same(_run(co, degree, WIN3, block=block, polish_warps=pw, ring_slots=slots), ref)


@pytest.mark.parametrize("degree", [2, 6, 9, 12])
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_compensated_polish_bit_identical_to_one_role_kernel(dev, degree, dtype):
    """The FP32-pipe compensated polish (RD_POLISH_DF) in the warp-specialised
    form: the same bits as its one-role form, for both storage types."""
    n = 4000 + 13 * degree
    co = to_soa(WL.gaussian(300 + degree, n, degree), dev, dtype)
    ref = _run(co, degree, WIN3, polish_mode="df")
    shapes = [(512, 6, 0), (256, 3, 4), (64, 1, 2)] if degree <= 6 else [(256, 3, 0), (128, 1, 2)]
    for block, pw, slots in shapes:
        _same(_run(co, degree, WIN3, polish_mode="df", block=block, polish_warps=pw, ring_slots=slots), ref)


def test_compensated_polish_littlewood_subsample_matches_oracle(dev, orc):
    """2^14 polynomials i = 4096 k of the 2^26 Littlewood batch through the
    warp-specialised compensated polish against the FP64 oracle at 1e-9."""
    idx = np.arange(1 << 14, dtype=np.uint64) * np.uint64(4096)
    co = WL.littlewood(2, idx)
    roots, status, _, st = _run(to_soa(co, dev, torch.complex64), 6, WIN2, block=512, polish_warps=6,
                                polish_mode="df")
    ref, ref_status, _, _ = orc.solve(co.astype(np.complex128), tol=1e-13)
    s = status.cpu().numpy()
    ok = (s == 0) & (ref_status == 0)
    assert ok.mean() > 0.999
    check_rejected(co.astype(np.complex128), s, ref, orc)
    compare_roots(roots.cpu().numpy().T[ok], ref[ok], co[ok].astype(np.complex128), orc, 1e-9, 1e3)
    assert st["wait_timeouts"] == 0


@pytest.mark.parametrize("ctas_per_sm", [1, 2])
def test_grid_smaller_than_the_sm_count_and_explicit_ctas(dev, ctas_per_sm):
    """ctas_per_sm fixed, and batches with fewer tasks than CTAs."""
    for n in (32 * 7 + 5, 1 << 18):
        co = WL.littlewood_soa_torch(2, 777, n, dev)
        ref = _run(co, 6, WIN2)
        got = _run(co, 6, WIN2, block=256, polish_warps=2, ctas_per_sm=ctas_per_sm)
        _same(got, ref)


def test_tile_clip_bit_identical(dev):
    """The full pipeline's own-tile clip (centres, radius, tile grid) runs in
    the polish warps exactly as in the one-role kernel."""
    nx, ny = 96, 54
    tiles = api.Window(-4.0, 4.0, -2.25, 2.25)
    centres, rho, _, _ = WL.tiles(-4.0, 4.0, -2.25, 2.25, nx, ny)
    co = to_soa(WL.gaussian(31, nx * ny, 6) * 1e-2, dev, torch.complex128)
    cen = torch.from_numpy(np.ascontiguousarray(centres)).to(dev)
    clip = api.make_clip(cen, float(rho), nx, ny, tiles)

    def run(**kw):
        p = api.params("mixed", **kw)
        hist = api.new_hist(W, H, dev)
        stats = api.new_stats(dev)
        api.roots_density(co, WIN3, hist, "mixed", p, clip=clip, stats=stats)
        torch.cuda.synchronize()
        return hist, api.stats_dict(stats)

    h0, s0 = run()
    h1, s1 = run(block=512, polish_warps=4)
    assert torch.equal(h0, h1) and s0 == s1 and s0["clipped"] > 0


def test_histogram_only_without_optional_outputs(dev):
    """roots, status and stats are optional: the histogram alone, as the
    benchmark's zero-copy leg asks for it, equals the one-role kernel's."""
    co = WL.littlewood_soa_torch(2, 5, 70001, dev)
    hists = []
    for kw in ({}, dict(block=512, polish_warps=10)):
        hist = api.new_hist(W, H, dev)
        api.roots_density(co, WIN2, hist, "mixed", api.params("mixed", **kw))
        torch.cuda.synchronize()
        hists.append(hist)
    assert torch.equal(hists[0], hists[1]) and int(hists[0].sum()) > 0


def test_graph_replay_bit_identical(dev):
    n = 1 << 16
    co = WL.littlewood_soa_torch(2, 99, n, dev)
    ref = _run(co, 6, WIN2)
    p = api.params("mixed", block=512, polish_warps=4)
    roots = torch.empty((6, n), dtype=torch.complex128, device=dev)
    status = torch.empty(n, dtype=torch.uint8, device=dev)
    hist = api.new_hist(W, H, dev)
    stats = api.new_stats(dev)
    # first launch outside the capture (it raises the kernel's shared-memory limit)
    api.roots_density(co, WIN2, hist, "mixed", p, roots=roots, status=status, stats=stats)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            api.hist_clear(hist)
            stats.zero_()
            api.roots_density(co, WIN2, hist, "mixed", p, roots=roots, status=status, stats=stats)
    for _ in range(3):
        roots.zero_()
        g.replay()
    torch.cuda.synchronize()
    _same((roots, status, hist, api.stats_dict(stats)), ref)


def test_littlewood_subsample_matches_oracle(dev, orc):
    """2^14 polynomials i = 4096 k of the 2^26 Littlewood batch against the
    FP64 oracle at the mixed path's 1e-9 bar."""
    idx = np.arange(1 << 14, dtype=np.uint64) * np.uint64(4096)
    co = WL.littlewood(2, idx)
    roots, status, _, st = _run(to_soa(co, dev, torch.complex64), 6, WIN2, block=512, polish_warps=4)
    ref, ref_status, _, _ = orc.solve(co.astype(np.complex128), tol=1e-13)
    s = status.cpu().numpy()
    ok = (s == 0) & (ref_status == 0)
    assert ok.mean() > 0.999
    check_rejected(co.astype(np.complex128), s, ref, orc)
    r = roots.cpu().numpy().T
    compare_roots(r[ok], ref[ok], co[ok].astype(np.complex128), orc, 1e-9, 1e3)
    assert st["polys"] == idx.size and st["wait_timeouts"] == 0


def test_bounded_wait_runs_out_and_reports(dev):
    """Every warp in the polish role: nothing fills the ring, each CTA's first
    wait ends after about 2 s, the abort flag stops the rest, and every
    polynomial comes back REJECTED and counted; the context stays usable."""
    n = 1000
    co = WL.littlewood_soa_torch(2, 0, n, dev)
    status = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    stats = api.new_stats(dev)
    t0 = time.perf_counter()
    api.N.call("rd_ws_selftest_timeout", api._ptr(co), n, api._ptr(status), api._ptr(stats), api._stream())
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st = api.stats_dict(stats)
    assert torch.all(status == 2)
    assert st["wait_timeouts"] == n and st["polys"] == n and st["status_rejected"] == n
    assert 1.5 <= dt <= 30.0, dt
    # the context still solves
    ref = _run(co, 6, WIN2)
    _same(_run(co, 6, WIN2, block=256, polish_warps=2), ref)


def test_autograd_roots_with_a_warp_specialised_shape(dev):
    """api.roots(..., params_) forwards the launch shape: the same roots, and
    so the same adjoint gradients, bit for bit."""
    co = to_soa(WL.gaussian(9, 20001, 6), dev, torch.complex128)
    grads = []
    for p in (None, api.params("mixed", block=512, polish_warps=10)):
        c = co.clone().requires_grad_(True)
        z, _ = api.roots(c, "mixed", p)
        (z.real ** 2 + z.imag ** 2).sum().backward()
        grads.append((z.detach(), c.grad))
    assert torch.equal(torch.view_as_real(grads[0][0]), torch.view_as_real(grads[1][0]))
    assert torch.equal(torch.view_as_real(grads[0][1]), torch.view_as_real(grads[1][1]))


@pytest.mark.parametrize("kw", [dict(), dict(max_iters=1), dict(polish_steps=0, polish_extra=0),
                                dict(residual_tol=1e-30, polish_extra=2), dict(collapse_tol=1.0),
                                dict(shift="rayleigh", exc_period=3), dict(polish_steps=1, polish_extra=0)])
def test_every_status_branch_bit_identical(dev, kw):
    """Degenerate rows (NaN, infinite and zero-leading coefficients) and
    parameter sets that drive NOT_CONVERGED (one sweep per level), no polish,
    REJECTED by the residual or the separation check: the warp-specialised
    kernel reproduces the one-role kernel's roots, status and counters."""
    n = 9001
    c = WL.gaussian(77, n, 6).astype(np.complex64)
    c[5, 2] = np.nan
    c[40, 6] = 0.0
    c[41, :] = 0.0
    c[700, 0] = np.inf
    c[8999, 6] = 0.0
    co = to_soa(c.astype(np.complex128), dev, torch.complex64)
    ref = _run(co, 6, WIN3, **kw)
    got = _run(co, 6, WIN3, block=512, polish_warps=10, **kw)
    # NaN roots compare by bits, so degenerate rows must match exactly too
    _same(got, ref)
    st = ref[3]
    assert st["status_degenerate"] == 5
    if kw.get("max_iters") == 1:
        assert st["status_not_converged"] > 0
    if kw.get("residual_tol") == 1e-30:
        assert st["status_rejected"] > 0
    if kw.get("collapse_tol") == 1.0:  # a tolerance far above the screen's 1e-4 floor is honoured
        assert st["status_rejected"] > n // 10
