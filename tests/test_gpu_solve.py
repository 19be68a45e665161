"""GPU parity: the CUDA solver and binning against the FP64 CPU oracle.

All inputs come from the seeded generators in paper_2507_02164_gb300.workloads;
expected values come from the oracle only.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2507_02164_gb300 import api, workloads as WL
from tests.gpu_common import (check_rejected, compare_roots, edge_distance, hist_np, matched, require_gpu,
                              roots_poly_major, to_soa)

pytestmark = pytest.mark.gpu

WIN1 = api.Window(-1.5, 1.5, -0.84375, 0.84375)
WIN2 = api.Window(-2.0, 2.0, -1.125, 1.125)
W, H = 1920, 1080
PLAIN_TOL, MIXED_TOL = 1e-11, 1e-9
# a root is held to the bar where the oracle's own deflation error,
# up to ~10 kappa 1e-13, is below it (plain: kappa <= 100, mixed: kappa <= 1000)
KAPPA_PLAIN, KAPPA_MIXED = 100.0, 1e3
# the mixed path may flag a few ill-conditioned polynomials as REJECTED
MAX_REJECTED = 2e-3


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _solve(coeffs_t, mode, window=None, **kw):
    d, n = coeffs_t.shape[0] - 1, coeffs_t.shape[1]
    roots = torch.empty((d, n), dtype=torch.complex128, device=coeffs_t.device)
    status = torch.empty(n, dtype=torch.uint8, device=coeffs_t.device)
    stats = api.new_stats(coeffs_t.device)
    p = api.params(mode, **kw)
    if window is None:
        api.roots_batched(coeffs_t, mode=mode, params_=p, roots=roots, status=status, stats=stats)
        hist = None
    else:
        hist = api.new_hist(W, H, coeffs_t.device)
        api.roots_density(coeffs_t, window, hist, mode=mode, params_=p, roots=roots, status=status, stats=stats)
    torch.cuda.synchronize()
    return roots_poly_major(roots), status.cpu().numpy(), hist, api.stats_dict(stats)


# ------------------------------------------------ plain FP64, known roots (C1)

@pytest.mark.parametrize("mode,tol,kcap", [("plain", PLAIN_TOL, KAPPA_PLAIN), ("mixed", MIXED_TOL, KAPPA_MIXED)])
def test_unit_disk_batch_matches_oracle_and_true_roots(dev, orc, mode, tol, kcap):
    """65,536 monic degree-6 polynomials from seeded roots in the unit disk."""
    n = 65536
    co, true_roots = WL.unit_disk_roots(1, n)
    roots, status, hist, st = _solve(to_soa(co, dev), mode, WIN1)
    ref, ref_status, _, _ = orc.solve(co, tol=1e-13)
    assert np.all(ref_status == 0)
    assert np.all(status != 1) and np.all(status != 3)
    if mode == "plain":
        assert np.all(status == 0)
    rejected = status == 2
    assert rejected.mean() <= MAX_REJECTED, int(rejected.sum())
    ok = ~rejected
    s_or, g = compare_roots(roots[ok], ref[ok], co[ok], orc, tol, kcap)
    s_true, _ = compare_roots(roots[ok], true_roots[ok], co[ok], orc, tol, kcap)
    assert s_or["n_excluded"] < 0.06 * roots[ok].size, s_or
    # a rejected polynomial has an ill-conditioned root
    check_rejected(co, status, true_roots, orc)
    # histogram: the oracle's binning of the GPU roots is the GPU histogram, bit for bit
    h_gpu = hist_np(hist)
    h_or_gpu_roots, oow = orc.hist(roots, WIN1.tuple(), W, H)
    assert np.array_equal(h_gpu, h_or_gpu_roots)
    assert st["binned"] == int(h_gpu.sum()) and st["out_of_window"] == oow
    assert st["binned"] + st["out_of_window"] == 6 * n and st["polys"] == n
    assert st["status_ok"] == int((status == 0).sum()) and st["status_rejected"] == int(rejected.sum())
    # against the oracle's own roots: differences only where a root sits within
    # 1e-9 of a pixel edge, or belongs to a polynomial flagged REJECTED
    h_or, _ = orc.hist(ref, WIN1.tuple(), W, H)
    diff = np.argwhere(h_gpu != h_or)
    near_edge = edge_distance(ref.reshape(-1), WIN1.tuple(), W, H) <= 1e-9
    explained = int(near_edge.sum()) + 6 * int(rejected.sum())
    assert np.abs(h_gpu.astype(np.int64) - h_or).sum() <= 2 * explained, diff[:10]


# ------------------------------------------------- Littlewood subsample (C2)

@pytest.mark.parametrize("mode,tol,kcap", [("mixed", MIXED_TOL, KAPPA_MIXED), ("plain", PLAIN_TOL, KAPPA_PLAIN)])
def test_littlewood_subsample_matches_oracle(dev, orc, mode, tol, kcap):
    """The 2^16 polynomials i = 1024 k of the 2^26 Littlewood batch."""
    idx = np.arange(1 << 16, dtype=np.uint64) * np.uint64(1024)
    co = WL.littlewood(2, idx)
    roots, status, hist, st = _solve(to_soa(co, dev, torch.complex64), mode, WIN2)
    ref, ref_status, _, _ = orc.solve(co.astype(np.complex128), tol=1e-13)
    assert np.all(ref_status == 0)
    assert (status == 0).mean() >= 1 - MAX_REJECTED, np.bincount(status, minlength=4)
    assert np.all((status == 0) | (status == 2))
    check_rejected(co.astype(np.complex128), status, ref, orc)
    ok = status == 0
    s, _ = compare_roots(roots[ok], ref[ok], co[ok].astype(np.complex128), orc, tol, kcap)
    h_gpu = hist_np(hist)
    h_ref, _ = orc.hist(roots, WIN2.tuple(), W, H)
    assert np.array_equal(h_gpu, h_ref)


# -------------------------------------------------- every degree, both modes

@pytest.mark.parametrize("degree", list(range(1, 13)))
@pytest.mark.parametrize("mode", ["mixed", "plain"])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("lanes", [1, 2])
def test_every_degree_matches_oracle(dev, orc, degree, mode, dtype, lanes):
    n = 1000 + 37  # several warps and a ragged tail
    co = WL.gaussian(100 + degree, n, degree)
    if dtype == torch.complex64:
        co = co.astype(np.complex64).astype(np.complex128)  # the stored values
    roots, status, _, st = _solve(to_soa(co, dev, dtype), mode, lanes=lanes)
    ref, ref_status, _, _ = orc.solve(co, tol=1e-13)
    good = (status == 0) & (ref_status == 0)
    assert good.mean() > 0.99, np.bincount(status, minlength=4)
    check_rejected(co, status, ref, orc)
    tol, kcap = (MIXED_TOL, KAPPA_MIXED) if mode == "mixed" else (PLAIN_TOL, KAPPA_PLAIN)
    compare_roots(roots[good], ref[good], co[good], orc, tol, kcap)
    assert st["polys"] == n


# ----------------------------------------------------------------- edge cases

def test_empty_batch_is_noop(dev):
    co = torch.zeros((7, 0), dtype=torch.complex64, device=dev)
    r, s = api.roots_batched(co, mode="mixed")
    assert r.shape == (6, 0) and s.shape == (0,)


@pytest.mark.parametrize("mode", ["mixed", "plain"])
def test_degenerate_inputs(dev, orc, mode):
    co = WL.gaussian(7, 40, 6)
    co[3, 6] = 0.0              # zero leading coefficient
    co[5, 2] = np.nan           # NaN coefficient
    co[7, 0] = np.inf           # infinite coefficient
    co[9, :] = 0.0              # zero polynomial
    roots, status, hist, st = _solve(to_soa(co, dev), mode, WIN1)
    bad = [3, 5, 7, 9]
    assert np.all(status[bad] == 3)
    assert np.all(np.isnan(roots[bad]))
    others = np.setdiff1d(np.arange(40), bad)
    assert np.all(status[others] != 3)
    assert st["status_degenerate"] == 4
    assert st["binned"] + st["out_of_window"] == 6 * 40
    assert st["out_of_window"] >= 4 * 6


def test_single_polynomial_and_degree_one(dev):
    co = np.array([[2 + 1j, 4 - 2j]])
    roots, status, _, _ = _solve(to_soa(co, dev), "plain")
    assert status[0] == 0 and abs(roots[0, 0] - (-(2 + 1j) / (4 - 2j))) < 1e-15


def test_max_iters_one_flags_not_converged(dev):
    co = WL.gaussian(8, 200, 6)
    _, status, _, st = _solve(to_soa(co, dev), "plain", max_iters=1)
    assert (status == 1).mean() > 0.9
    assert st["status_not_converged"] == int((status == 1).sum())


def test_rayleigh_shift_with_exceptional_shift_also_converges(dev, orc):
    idx = np.arange(4096, dtype=np.uint64)
    co = WL.littlewood(2, idx)
    roots, status, _, _ = _solve(to_soa(co, dev, torch.complex64), "mixed", shift="rayleigh", exc_period=10)
    ref, _, _, _ = orc.solve(co.astype(np.complex128))
    ok = status == 0
    assert ok.mean() > 0.999
    check_rejected(co.astype(np.complex128), status, ref, orc)
    compare_roots(roots[ok], ref[ok], co[ok].astype(np.complex128), orc, MIXED_TOL, KAPPA_MIXED)


def test_launch_shapes_give_identical_results(dev):
    """Block size and grid only change the schedule, never the arithmetic."""
    co = to_soa(WL.littlewood(2, 5000), dev, torch.complex64)
    base, bst, _, _ = _solve(co, "mixed")
    for block, cps in ((32, 1), (64, 3), (256, 2)):
        r, s, _, _ = _solve(co, "mixed", block=block, ctas_per_sm=cps)
        assert np.array_equal(r, base) and np.array_equal(s, bst)


@pytest.mark.parametrize("mode,tol,kcap", [("plain", PLAIN_TOL, KAPPA_PLAIN), ("mixed", MIXED_TOL, KAPPA_MIXED)])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_roots_at_zero(dev, orc, mode, tol, kcap, k):
    """p(z) = z^k q(z) (a_0 = .. = a_{k-1} = 0 exactly, q of degree 6 - k with
    complex-Gaussian coefficients). k = 1: a simple zero root, held to the
    bar with the others. k >= 2: a k-fold zero. Newton's method converges to
    it only linearly, so the mixed path's FP64 residual check fails and the
    polynomial is REJECTED (the condition number as the oracle defines it
    stays O(1) at a multiple root, so the rule that a rejected polynomial has
    a root with kappa > 100 does not apply here). The plain path returns the
    k copies within the eigenvalue perturbation bound eps^(1/k) of 0, and q's
    roots within 1e-9 of the oracle's (beside the zero cluster the FP64
    eigenvalue computation of both carries the cluster's splitting into its
    rounding: measured up to 7e-10 relative to kappa)."""
    g = np.random.default_rng(40 + k)
    n = 4096
    co = np.zeros((n, 7), dtype=np.complex128)
    co[:, k:] = g.standard_normal((n, 7 - k)) + 1j * g.standard_normal((n, 7 - k))
    roots, status, _, _ = _solve(to_soa(co, dev), mode)
    ref, ref_status, _, _ = orc.solve(co, tol=1e-13)
    assert np.all(status != 1) and np.all(status != 3)
    if k == 1:
        check_rejected(co, status, ref, orc)
        ok = status == 0
        assert ok.mean() >= 1 - MAX_REJECTED
        compare_roots(roots[ok], ref[ok], co[ok], orc, tol, kcap)
        assert np.abs(roots[ok]).min(axis=1).max() <= tol
        return
    if mode == "mixed":
        assert np.all(status == 2), np.bincount(status, minlength=4)
        return
    assert np.all(status == 0)
    by_size = lambda z: np.take_along_axis(z, np.argsort(np.abs(z), axis=1), axis=1)
    g_, r = by_size(roots), by_size(ref)
    assert np.abs(g_[:, :k]).max() <= {2: 1e-6, 3: 1e-4}[k], float(np.abs(g_[:, :k]).max())
    gq = matched(g_[:, k:], r[:, k:])
    err = np.abs(gq - r[:, k:]) / np.maximum(1.0, np.abs(r[:, k:]))
    assert err.max() <= 1e-9, float(err.max())


@pytest.mark.parametrize("mode", ["mixed", "plain"])
@pytest.mark.parametrize("case", ["littlewood6", "real_gauss12", "complex_gauss9"])
def test_roots_do_not_depend_on_warp_mates(dev, mode, case):
    """A polynomial's roots are the same bits whichever polynomials share its
    warp (the sweep size is the warp's largest active block; a frozen lane's
    rotations are exact identities). Real coefficients included: their
    imaginary parts are signed zeros throughout the sweeps. The uneven path
    relies on this, as it packs each degree bin in an unspecified order."""
    g = np.random.default_rng(17)
    if case == "littlewood6":
        co = WL.littlewood(3, 1 << 15)
    elif case == "real_gauss12":
        co = g.standard_normal((1 << 13, 13)).astype(np.complex128)
    else:
        co = WL.gaussian(9, 1 << 13, 9)
    perm = g.permutation(co.shape[0])
    dt = torch.complex64 if mode == "mixed" else torch.complex128
    ra, sa, _, _ = _solve(to_soa(co, dev, dt), mode)
    rb, sb, _, _ = _solve(to_soa(co[perm], dev, dt), mode)
    assert np.array_equal(ra[perm].view(np.int64), rb.view(np.int64))
    assert np.array_equal(sa[perm], sb)


# -------------------------------------------------------- standalone binning

def test_density_accumulate_matches_oracle_bit_for_bit(dev, orc):
    g = np.random.default_rng(5)
    z = g.uniform(-1.7, 1.7, 300001) + 1j * g.uniform(-1.0, 1.0, 300001)
    # exact edges, corners, NaN and infinities
    z[:8] = [-1.5 + 0.84375j, 1.5 + 0j, -0.84375j, 1.5 - 0.84375j, complex(np.nan, 0), complex(0, np.inf),
             -1.5 - 0.84375j, 0j]
    t = torch.from_numpy(z).to(dev)
    hist = api.new_hist(W, H, dev)
    stats = api.new_stats(dev)
    api.density_accumulate(t, WIN1, hist, stats=stats)
    api.density_accumulate(t[:1000], WIN1, hist, stats=stats)  # accumulates
    torch.cuda.synchronize()
    ref, oow = orc.hist(np.concatenate([z, z[:1000]]), WIN1.tuple(), W, H)
    assert np.array_equal(hist_np(hist), ref)
    st = api.stats_dict(stats)
    assert st["out_of_window"] == oow and st["binned"] == int(ref.sum())


def test_hist_clear_zeroes_odd_sizes(dev):
    for words in (1, 3, 5, 1920 * 1080, 1920 * 1080 + 3):
        buf = torch.full((words + 8,), -1, dtype=torch.int32, device=dev)
        api.N.call("rd_hist_clear", api._ptr(buf[1:]), words, api._stream())
        torch.cuda.synchronize()
        b = buf.cpu().numpy()
        assert b[0] == -1 and np.all(b[1:words + 1] == 0) and np.all(b[words + 1:] == -1)


# ------------------------------------------ the paper's fixed schedule (Alg. 2)

def test_paper_fixed_schedule_fp32_matches_oracle_fixed_schedule(dev, orc):
    """T = 10 sweeps per eigenvalue, Rayleigh shift, FP32, no polish (the
    paper's settings, Sec. IV): exactly (d-1) T sweeps per polynomial, and
    where the FP64 fixed schedule converged the FP32 GPU roots agree with it
    to FP32 accuracy."""
    from tests.helpers import matched_errors
    n = 4096 + 7
    co, true_roots = WL.unit_disk_roots(1, n)
    co32 = co.astype(np.complex64).astype(np.complex128)
    roots, status, _, st = _solve(to_soa(co32, dev, torch.complex64), "mixed", fixed_sweeps=10, shift="rayleigh",
                                  exc_period=0, polish_steps=0, polish_extra=0)
    assert np.all(status == 0)
    assert st["sweeps"] == n * 5 * 10 and st["newton_steps"] == 0
    ref, _ = orc.solve_fixed(co32, T=10)
    converged = matched_errors(ref, true_roots).max(axis=1) < 1e-6
    # the fixed schedule leaves ~18 % of these polynomials with a root off by > 1e-6 (oracle pin)
    assert converged.mean() > 0.75
    err = matched_errors(roots[converged], ref[converged])
    kappa = orc.root_condition(co32[converged], ref[converged])
    assert (err <= 1e-5 * np.maximum(1.0, kappa)).mean() > 0.99


# ------------------------------------------------ double-float polish variant

@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_double_float_polish_matches_oracle(dev, orc, dtype):
    """RD_POLISH_DF: Newton steps in double-float arithmetic, FP64 final check;
    same 1e-9 bar as the FP64 polish, on the unit-disk and Littlewood batches."""
    co, true_roots = WL.unit_disk_roots(1, 65536)
    if dtype == torch.complex64:
        co = co.astype(np.complex64).astype(np.complex128)
    roots, status, hist, st = _solve(to_soa(co, dev, dtype), "mixed", WIN1, polish_mode="df")
    ref, _, _, _ = orc.solve(co, tol=1e-13)
    assert np.all((status == 0) | (status == 2)) and (status == 2).mean() <= MAX_REJECTED
    check_rejected(co, status, ref, orc)
    ok = status == 0
    compare_roots(roots[ok], ref[ok], co[ok], orc, MIXED_TOL, KAPPA_MIXED)
    h_ref, _ = orc.hist(roots, WIN1.tuple(), W, H)
    assert np.array_equal(hist_np(hist), h_ref)
    idx = np.arange(1 << 16, dtype=np.uint64) * np.uint64(1024)
    cl = WL.littlewood(2, idx)
    roots, status, _, _ = _solve(to_soa(cl, dev, torch.complex64), "mixed", polish_mode="df")
    ref, _, _, _ = orc.solve(cl.astype(np.complex128))
    ok = status == 0
    assert ok.mean() >= 1 - MAX_REJECTED
    check_rejected(cl.astype(np.complex128), status, ref, orc)
    compare_roots(roots[ok], ref[ok], cl[ok].astype(np.complex128), orc, MIXED_TOL, KAPPA_MIXED)


# ------------------------------------- full size, in the benchmark's launch shape

@pytest.mark.parametrize("polish", ["fp64", "df"])
def test_full_littlewood_batch_sampled(dev, orc, polish):
    """The 2^26-polynomial Littlewood batch exactly as bench.py times it (fused
    roots + histogram, autotuned launch shape, mixed; the FP64 polish of the
    headline and the compensated FP32-pipe polish), with the roots stored:
    every counter adds up, the fused histogram equals the standalone binning
    of the stored roots, and 2^16 polynomials spread over the batch match the
    oracle at the 1e-9 bar (mixed) and, for the plain FP64 path on the same
    sample, at 1e-11."""
    from paper_2507_02164_gb300 import autotune
    n = 1 << 26
    coeffs = WL.littlewood_soa_torch(2, 0, n, dev)
    tuned = autotune.tune("mixed", degrees=[6], polish=polish)
    p = autotune.degree_params(tuned, 6, "mixed", polish)
    hist = api.new_hist(W, H, dev)
    stats = api.new_stats(dev)
    roots = torch.empty((6, n), dtype=torch.complex128, device=dev)
    status = torch.empty(n, dtype=torch.uint8, device=dev)
    api.roots_density(coeffs, WIN2, hist, mode="mixed", params_=p, roots=roots, status=status, stats=stats)
    torch.cuda.synchronize()
    st = api.stats_dict(stats)
    assert st["polys"] == n and st["binned"] + st["out_of_window"] == 6 * n
    h = hist_np(hist)
    assert int(h.sum(dtype=np.int64)) == st["binned"]
    h2 = api.new_hist(W, H, dev)
    api.density_accumulate(roots.reshape(-1), WIN2, h2)
    torch.cuda.synchronize()
    assert np.array_equal(hist_np(h2), h)
    s = status.cpu().numpy()
    assert np.all((s == 0) | (s == 2)) and (s == 2).mean() <= MAX_REJECTED
    idx = np.arange(1 << 16, dtype=np.int64) * 1024 + 511
    sample = torch.from_numpy(idx).to(dev)
    r_s = roots[:, sample].cpu().numpy().T
    co = coeffs[:, sample].cpu().numpy().T.astype(np.complex128)
    ref, ref_st, _, _ = orc.solve(co)
    check_rejected(co, s[idx], ref, orc)
    ok = (s[idx] == 0) & (ref_st == 0)
    compare_roots(r_s[ok], ref[ok], co[ok], orc, MIXED_TOL, KAPPA_MIXED)
    pr, ps = api.roots_batched(coeffs[:, sample].contiguous(), mode="plain")
    torch.cuda.synchronize()
    pr = pr.cpu().numpy().T
    okp = (ps.cpu().numpy() == 0) & (ref_st == 0)
    compare_roots(pr[okp], ref[okp], co[okp], orc, PLAIN_TOL, KAPPA_PLAIN)


@pytest.mark.parametrize("mode", ["mixed", "plain"])
@pytest.mark.parametrize("lanes", [1, 2])
def test_roots_do_not_depend_on_a_power_of_two_scale(dev, mode, lanes):
    """p and 2^e p have the same roots: complex128 coefficients far beyond the
    FP32 range (2^130, 2^600) or below it (2^-130) give bit-identical roots
    and statuses (the normalisation divides exactly scaled values; the mixed
    polish rescales before its FP32 copies)."""
    co = WL.gaussian(11, 4096 + 5, 8)
    r0, s0, _, _ = _solve(to_soa(co, dev), mode, lanes=lanes)
    assert (s0 == 0).mean() > 0.99
    for e in (130, -130, 600):
        r, s, _, _ = _solve(to_soa(co * 2.0 ** e, dev), mode, lanes=lanes)
        assert np.array_equal(r, r0) and np.array_equal(s, s0), e


def test_inputs_in_page_locked_host_memory_give_identical_results(dev):
    """Zero copy: coefficients in page-locked host memory are read by the
    kernel across the host link; roots, status and histogram equal those of
    the same coefficients on the device, bit for bit. Pageable host memory
    is refused before any kernel sees it."""
    co = to_soa(WL.gaussian(13, 20000 + 7, 6), dev, torch.complex64)
    host = co.cpu().pin_memory()
    r_d, s_d, h_d, st_d = _solve(co, "mixed", WIN2)
    hist = api.new_hist(W, H, dev)
    roots = torch.empty((6, co.shape[1]), dtype=torch.complex128, device=dev)
    status = torch.empty(co.shape[1], dtype=torch.uint8, device=dev)
    stats = api.new_stats(dev)
    api.roots_density(host, WIN2, hist, mode="mixed", roots=roots, status=status, stats=stats)
    torch.cuda.synchronize()
    assert np.array_equal(roots_poly_major(roots), r_d) and np.array_equal(status.cpu().numpy(), s_d)
    assert torch.equal(hist, h_d) and api.stats_dict(stats) == st_d
    r_b, s_b = api.roots_batched(host, mode="plain")
    r_c, s_c = api.roots_batched(co, mode="plain")
    torch.cuda.synchronize()
    assert r_b.is_cuda and torch.equal(r_b, r_c) and torch.equal(s_b, s_c)
    with pytest.raises(ValueError, match="page-locked"):
        api.roots_batched(co.cpu(), mode="mixed")


@pytest.mark.parametrize("window,W_,H_", [((-2.0, 2.0, -1.125, 1.125), 1920, 1080),
                                          ((-0.3, 1.7, -0.9, 0.2), 777, 333),
                                          ((1e6, 1e6 + 2.0, -1.0, 0.5), 1920, 1080)])
def test_binning_at_pixel_edges_matches_fp64_bit_for_bit(dev, orc, window, W_, H_):
    """The pixel index is taken in double-float with an FP64 fallback within
    1e-6 pixel of an edge; against the oracle's FP64 binning: random points,
    points on every kind of edge and 1..4 ulps beside them, far and non-finite
    points, and a window (the last) whose size disables the fast path."""
    g = np.random.default_rng(W_)
    xmin, xmax, ymin, ymax = window
    n = 200000
    pts = [g.uniform(xmin - 0.1 * (xmax - xmin), xmax, n) + 1j * g.uniform(ymin, ymax + 0.1 * (ymax - ymin), n)]
    ex = xmin + (xmax - xmin) * g.integers(0, W_ + 1, 5000) / W_  # pixel edges, as the host computes them
    ey = ymax - (ymax - ymin) * g.integers(0, H_ + 1, 5000) / H_
    def ulps(v, k):  # v moved by k ulps
        for _ in range(abs(k)):
            v = np.nextafter(v, np.inf if k > 0 else -np.inf)
        return v

    for k in range(-4, 5):
        pts.append(ulps(ex, k) + 1j * g.uniform(ymin, ymax, 5000) if k else ex + 1j * ey)
        pts.append(g.uniform(xmin, xmax, 5000) + 1j * (ulps(ey, k) if k else ey))
    pts.append(np.array([complex(np.nan, 0), complex(0, np.inf), complex(1e300, 0), complex(-1e200, 1e200)]))
    z = np.concatenate(pts)
    hist = api.new_hist(W_, H_, dev)
    api.density_accumulate(torch.from_numpy(z).to(dev), api.Window(*window), hist)
    torch.cuda.synchronize()
    ref, _ = orc.hist(z, window, W_, H_)
    assert np.array_equal(hist_np(hist), ref)
