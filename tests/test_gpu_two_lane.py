"""GPU parity of the two-lanes-per-polynomial solver (params.lanes = 2)
against the FP64 CPU oracle, and its bookkeeping against the one-lane solver.

Two lanes split the Hessenberg matrix by column parity and exchange the
rotations by warp shuffle; the arithmetic is the same QR iteration, so the
roots must meet the same bars as the one-lane solver, the counters must add
up per polynomial (not per lane), and the fixed schedule must run exactly
(d-1) T sweeps per polynomial. Expected values come from the oracle only.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2507_02164_gb300 import api, workloads as WL
from tests.gpu_common import check_rejected, compare_roots, hist_np, require_gpu, roots_poly_major, to_soa

pytestmark = pytest.mark.gpu

WIN2 = api.Window(-2.0, 2.0, -1.125, 1.125)
W, H = 1920, 1080
MIXED_TOL, KAPPA_MIXED = 1e-9, 1e3
PLAIN_TOL, KAPPA_PLAIN = 1e-11, 100.0


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _solve(coeffs_t, mode, window=None, **kw):
    d, n = coeffs_t.shape[0] - 1, coeffs_t.shape[1]
    roots = torch.empty((d, n), dtype=torch.complex128, device=coeffs_t.device)
    status = torch.empty(n, dtype=torch.uint8, device=coeffs_t.device)
    stats = api.new_stats(coeffs_t.device)
    p = api.params(mode, **kw)
    hist = None
    if window is None:
        api.roots_batched(coeffs_t, mode=mode, params_=p, roots=roots, status=status, stats=stats)
    else:
        hist = api.new_hist(W, H, coeffs_t.device)
        api.roots_density(coeffs_t, window, hist, mode=mode, params_=p, roots=roots, status=status, stats=stats)
    torch.cuda.synchronize()
    return roots_poly_major(roots), status.cpu().numpy(), hist, api.stats_dict(stats)


@pytest.mark.parametrize("degree", [2, 3, 7, 8, 11, 12])
@pytest.mark.parametrize("mode", ["mixed", "plain"])
def test_two_lanes_match_one_lane_counters_and_oracle(dev, orc, degree, mode):
    """Littlewood-like +-1 coefficients (unit-modulus roots near the circle)
    for odd and even degrees: roots within the mode's bar of the oracle, the
    histogram equal to the oracle's binning of the GPU roots, and counters per
    polynomial: polys, statuses, binned + out of window = d n."""
    n = 4096 + 9  # ragged over 16 polynomials per warp
    g = np.random.default_rng(700 + degree)
    co = g.choice([-1.0, 1.0], size=(n, degree + 1)).astype(np.complex128)
    co_t = to_soa(co, dev, torch.complex64)
    r2, s2, h2, st2 = _solve(co_t, mode, WIN2, lanes=2)
    r1, s1, _, st1 = _solve(co_t, mode, WIN2, lanes=1)
    ref, ref_st, _, _ = orc.solve(co)
    tol, kcap = (MIXED_TOL, KAPPA_MIXED) if mode == "mixed" else (PLAIN_TOL, KAPPA_PLAIN)
    # +-1 polynomials of low degree often have a double root ((z-1)^2 (z+1)
    # at degree 3): the mixed path rejects those, with one lane or two alike
    assert (s1 == s2).mean() > 0.995, (np.bincount(s1, minlength=4), np.bincount(s2, minlength=4))
    ok = (s2 == 0) & (ref_st == 0)
    assert ok.mean() > 0.5, np.bincount(s2, minlength=4)
    check_rejected(co, s1, ref, orc)
    check_rejected(co, s2, ref, orc)
    compare_roots(r2[ok], ref[ok], co[ok], orc, tol, kcap)
    h_ref, oow = orc.hist(r2, WIN2.tuple(), W, H)
    assert np.array_equal(hist_np(h2), h_ref)
    assert st2["polys"] == n == st1["polys"]
    assert st2["binned"] == int(h_ref.sum()) and st2["out_of_window"] == oow
    assert st2["binned"] + st2["out_of_window"] == degree * n
    for k, v in ((0, "status_ok"), (1, "status_not_converged"), (2, "status_rejected"), (3, "status_degenerate")):
        assert st2[v] == int((s2 == k).sum()), v
    # sweeps and rotations counted once per polynomial: within a few % of one lane
    assert abs(st2["sweeps"] - st1["sweeps"]) <= 0.05 * st1["sweeps"]
    assert st2["rotations"] <= st2["sweeps"] * (degree - 1)
    if mode == "mixed":
        assert st2["newton_steps"] >= 3 * degree * int((s2 != 3).sum()) * 0.99


@pytest.mark.parametrize("degree", [7, 12])
def test_two_lanes_fixed_schedule_counts_exactly(dev, degree):
    """Alg. 2's fixed schedule: exactly (d-1) T sweeps per polynomial and the
    pair-summed rotation and pair counts of a full schedule."""
    n = 1000 + 3
    co = WL.gaussian(50 + degree, n, degree)
    T = 6
    _, status, _, st = _solve(to_soa(co, dev, torch.complex64), "mixed", lanes=2, fixed_sweeps=T,
                              shift="rayleigh", exc_period=0, polish_steps=0, polish_extra=0)
    assert np.all(status == 0)
    assert st["sweeps"] == n * (degree - 1) * T
    # active size m = d, d-1, .., 2, T sweeps each: m - 1 rotations, m (m+1) - 2 pair updates
    ms = np.arange(2, degree + 1)
    assert st["rotations"] == n * T * int((ms - 1).sum())
    assert st["pair_updates"] == n * T * int((ms * (ms + 1) - 2).sum())
    assert st["newton_steps"] == 0


@pytest.mark.parametrize("degree", [7, 12])
@pytest.mark.parametrize("mode", ["mixed", "plain"])
def test_two_lanes_degenerate_inputs(dev, degree, mode):
    co = WL.gaussian(9, 40, degree)
    co[3, degree] = 0.0
    co[5, 2] = np.nan
    co[7, 0] = np.inf
    co[9, :] = 0.0
    roots, status, hist, st = _solve(to_soa(co, dev), mode, WIN2, lanes=2)
    bad = [3, 5, 7, 9]
    assert np.all(status[bad] == 3)
    assert np.all(np.isnan(roots[bad]))
    others = np.setdiff1d(np.arange(40), bad)
    assert np.all(status[others] != 3)
    assert np.all(np.isfinite(roots[others]))
    assert st["status_degenerate"] == 4 and st["polys"] == 40
    assert st["binned"] + st["out_of_window"] == degree * 40


def test_two_lanes_rayleigh_shift_with_exceptional_shift(dev, orc):
    co = WL.gaussian(31, 2048 + 5, 10)
    roots, status, _, _ = _solve(to_soa(co, dev), "mixed", lanes=2, shift="rayleigh", exc_period=10)
    ref, ref_st, _, _ = orc.solve(co)
    ok = (status == 0) & (ref_st == 0)
    assert ok.mean() > 0.99
    check_rejected(co, status, ref, orc)
    compare_roots(roots[ok], ref[ok], co[ok], orc, MIXED_TOL, KAPPA_MIXED)


def test_two_lanes_launch_shapes_give_identical_results(dev):
    co = to_soa(WL.gaussian(12, 5000, 12), dev, torch.complex64)
    base, bst, _, _ = _solve(co, "mixed", lanes=2)
    for block, cps in ((32, 1), (64, 3), (256, 1)):
        r, s, _, _ = _solve(co, "mixed", lanes=2, block=block, ctas_per_sm=cps)
        assert np.array_equal(r, base) and np.array_equal(s, bst)


def test_lanes_two_with_double_float_polish_is_refused(dev):
    co = to_soa(WL.gaussian(1, 64, 10), dev, torch.complex64)
    with pytest.raises(api.N.RootDensityError, match="lanes"):
        _solve(co, "mixed", lanes=2, polish_mode="df")
    with pytest.raises(api.N.RootDensityError, match="lanes"):
        _solve(co, "mixed", lanes=3)


@pytest.mark.parametrize("lanes", [1, 2])
def test_uneven_batch_two_lanes_matches_oracle(dev, orc, lanes):
    """The uneven-degree path (degrees 1..12) with both solver layouts."""
    n = 12000 + 11
    packed, deg, off = WL.uneven_gaussian(5, n, dtype=np.complex64)
    c_t = torch.from_numpy(packed).to(dev)
    d_t = torch.from_numpy(deg).to(dev)
    o_t = torch.from_numpy(off).to(dev)
    ws = api.new_uneven_workspace(n, packed.size, torch.complex64, dev)
    stats = api.new_stats(dev)
    roots, status = api.roots_uneven(c_t, d_t, o_t, ws, mode="mixed", params_=api.params("mixed", lanes=lanes),
                                     stats=stats)
    torch.cuda.synchronize()
    r = roots.cpu().numpy()
    s = status.cpu().numpy()
    pk = packed.astype(np.complex128)
    assert np.all((s == 0) | (s == 2)) and (s == 2).mean() <= 2e-3
    for d in np.unique(deg):
        idx = np.nonzero(deg == d)[0]
        rows = np.stack([pk[off[i]:off[i + 1]] for i in idx])
        rg = np.stack([r[off[i] - i: off[i] - i + d] for i in idx])
        ref, ref_st, _, _ = orc.solve(rows)
        good = (s[idx] == 0) & (ref_st == 0)
        assert good.mean() > 0.99, (d, good.mean())
        check_rejected(rows, s[idx], ref, orc)
        compare_roots(rg[good], ref[good], rows[good], orc, MIXED_TOL, KAPPA_MIXED)
    st = api.stats_dict(stats)
    assert st["polys"] == n and st["status_ok"] == int((s == 0).sum())


@pytest.mark.parametrize("degree", [6, 11])
def test_two_lanes_honour_a_large_collapse_tolerance(dev, degree):
    """collapse_tol far above the FP32 screen's 1e-4 floor: the pair of lanes
    rejects exactly the polynomials one lane rejects, and many of them."""
    co = to_soa(WL.gaussian(123 + degree, 4001, degree), dev, torch.complex128)
    _, s1, _, _ = _solve(co, "mixed", lanes=1, collapse_tol=1.0)
    _, s2, _, _ = _solve(co, "mixed", lanes=2, collapse_tol=1.0)
    assert np.array_equal(s1, s2) and (s1 == 2).sum() > 400
