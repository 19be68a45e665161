"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test states what fixes the expected value: a closed form, an invariant,
a library routine (LAPACK through numpy, mpmath at high precision, numpy's
Gauss-Legendre rule and histogram), or a number the paper prints.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

from paper_2507_02164_gb300 import workloads as W
from tests.helpers import match, matched_errors, rel_err

EPS = 2.0 ** -53
TOL = 1e-13                # deflation tolerance of the plain FP64 configuration
DEFL_BOUND = 50 * TOL      # root error per unit of condition number it may cause
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed):
    return np.random.default_rng(seed)


def crandn(g, *shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def random_hessenberg(g, n):
    A = crandn(g, n, n)
    return np.triu(A, -1)


# ------------------------------------------------------------- Givens (Sec. II-C)

def test_givens_zeroes_second_component(orc):
    g = rng(1)
    for _ in range(200):
        a, b = crandn(g, 2) * 10.0 ** g.uniform(-5, 5)
        c, s = orc.givens(a, b)
        G = np.array([[c, s], [-np.conj(s), np.conj(c)]])
        v = G @ np.array([a, b])
        r = math.hypot(abs(a), abs(b))
        assert abs(v[0] - r) <= 4 * EPS * r
        assert abs(v[1]) <= 4 * EPS * r
        assert np.allclose(G @ G.conj().T, np.eye(2), atol=16 * EPS, rtol=0)


def test_givens_zero_pair_and_zero_b(orc):
    c, s = orc.givens(0.0, 0.0)
    assert (c, s) == (1.0, 0.0)
    c, s = orc.givens(3 - 4j, 0.0)
    assert abs(c * (3 - 4j) - 5.0) < 1e-15 and s == 0.0
    c, s = orc.givens(0.0, 2j)
    assert c == 0.0 and abs(s * 2j - 2.0) < 1e-15


# --------------------------------------------------- companion matrix (Sec. II-B)

def test_companion_characteristic_polynomial(orc):
    g = rng(2)
    for n in (1, 2, 5, 6, 12):
        b = crandn(g, n)
        A = orc.companion(b)
        # np.poly: characteristic polynomial from LAPACK eigenvalues, highest power first
        charp = np.poly(A)[::-1]
        assert np.allclose(charp, np.concatenate([b, [1.0]]), atol=1e-10 * (1 + np.abs(b).sum()))
        assert np.allclose(np.tril(A, -2), 0)


# ------------------------------------------ one shifted sweep (Alg. 2, Appendix A)

@pytest.mark.parametrize("n,m", [(8, 8), (8, 5), (6, 6), (2, 2), (12, 12)])
def test_sweep_keeps_hessenberg_trace_and_spectrum(orc, n, m):
    g = rng(3 + n + m)
    A = random_hessenberg(g, n)
    s = complex(crandn(g, 1)[0])
    B = orc.qr_sweep(A, m, s)
    norm = np.linalg.norm(A)
    # Appendix A: the sweep keeps the Hessenberg form (only rounding below the subdiagonal)
    assert np.abs(np.tril(B, -2)).max() <= 16 * EPS * norm
    # entries outside the leading m x m block are not touched
    assert np.array_equal(B[m:, :], A[m:, :]) and np.array_equal(B[:, m:], A[:, m:])
    # a unitary similarity on the active block: trace and spectrum are preserved
    blkA, blkB = A[:m, :m], B[:m, :m]
    assert abs(np.trace(blkA) - np.trace(blkB)) <= 64 * EPS * norm * m
    ea = np.linalg.eigvals(blkA)
    eb = np.linalg.eigvals(blkB)
    assert np.abs(match(ea, eb) - ea).max() <= 1e-10 * norm
    # Frobenius norm preserved (unitary similarity)
    assert abs(np.linalg.norm(blkA) - np.linalg.norm(blkB)) <= 64 * EPS * norm * m


def test_sweep_equals_rq_of_lapack_qr(orc):
    """A - sI = QR (LAPACK Householder QR), then RQ + sI. The Givens QR of a
    Hessenberg matrix differs from LAPACK's only by a diagonal unitary D
    (Q -> Q D, R -> D^H R), which changes RQ by the similarity D^H (RQ) D: the
    moduli of all entries and the diagonal are unchanged."""
    g = rng(7)
    for n in (3, 6, 9):
        A = random_hessenberg(g, n)
        s = complex(crandn(g, 1)[0])
        Q, R = np.linalg.qr(A - s * np.eye(n))
        ref = R @ Q + s * np.eye(n)
        got = orc.qr_sweep(A, n, s)
        scale = np.linalg.norm(A)
        assert np.abs(np.abs(got) - np.abs(ref)).max() <= 1e-13 * scale
        assert np.abs(np.diag(got) - np.diag(ref)).max() <= 1e-13 * scale


def test_wilkinson_shift_is_nearer_eigenvalue(orc):
    g = rng(8)
    for _ in range(100):
        A = random_hessenberg(g, 5)
        mu = orc.wilkinson_shift(A, 5)
        ev = np.linalg.eigvals(A[3:5, 3:5])
        best = ev[np.argmin(np.abs(ev - A[4, 4]))]
        assert abs(mu - best) <= 1e-12 * (1 + abs(best))


# ------------------------------------------------------------- whole solver

def test_roots_of_polynomials_built_from_known_roots(orc):
    """Degree-6 polynomials expanded from seeded roots in the unit disk: the
    oracle returns the seeded roots up to the root's condition number times
    the deflation tolerance."""
    coeffs, true_roots = W.unit_disk_roots(1, 4000)
    roots, status, sweeps, _ = orc.solve(coeffs, tol=1e-13)
    assert np.all(status == 0)
    err = matched_errors(roots, true_roots)
    kappa = orc.root_condition(coeffs, true_roots)
    # dropping a subdiagonal entry below tol * |diag| is a backward error of
    # order tol, amplified by the root's conditioning
    assert np.all(err <= DEFL_BOUND * np.maximum(1.0, kappa))
    assert np.median(err) < 1e-13
    assert 10 <= sweeps.mean() <= 40


@pytest.mark.parametrize("seed,kind", [(21, "gauss"), (22, "littlewood"), (23, "gauss12")])
def test_roots_match_lapack(orc, seed, kind):
    if kind == "gauss":
        co = W.gaussian(seed, 1500, 6)
    elif kind == "littlewood":
        co = W.littlewood(seed, 1500).astype(np.complex128)
    else:
        co = W.gaussian(seed, 300, 12)
    roots, status, _, _ = orc.solve(co)
    assert np.all(status == 0)
    ref = np.array([np.roots(c[::-1]) for c in co])
    kappa = orc.root_condition(co, ref)
    err = matched_errors(roots, ref)
    assert np.all(err <= DEFL_BOUND * np.maximum(1.0, kappa))


def test_roots_match_mpmath_high_precision(orc):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    co = W.gaussian(31, 60, 6)
    roots, status, _, _ = orc.solve(co)
    assert np.all(status == 0)
    for i, c in enumerate(co):
        ref = mpmath.polyroots([mpmath.mpc(x.real, x.imag) for x in c[::-1]], maxsteps=200, extraprec=120)
        ref = np.array([complex(r) for r in ref])
        kappa = orc.root_condition(co[i:i + 1], ref[None, :])[0]
        err = rel_err(match(ref, roots[i]), ref)
        assert np.all(err <= DEFL_BOUND * np.maximum(1.0, kappa)), (i, err, kappa)


def _stable_quadratic(b1, b0):
    sq = np.sqrt(complex(b1 * b1 - 4 * b0))
    if (np.conj(b1) * sq).real < 0:
        sq = -sq
    q = -0.5 * (b1 + sq)
    if q == 0:
        return np.array([0.0, 0.0], dtype=complex)
    return np.array([q, b0 / q])


def test_degree2_closed_form(orc):
    g = rng(9)
    co = crandn(g, 500, 3)
    roots, status, _, _ = orc.solve(co)
    assert np.all(status == 0)
    for i, c in enumerate(co):
        ref = _stable_quadratic(c[1] / c[2], c[0] / c[2])
        kappa = orc.root_condition(c[None, :], ref[None, :])[0]
        assert np.all(rel_err(match(ref, roots[i]), ref) <= DEFL_BOUND * np.maximum(1.0, kappa))


def _cardano(b2, b1, b0):
    """Roots of z^3 + b2 z^2 + b1 z + b0 by Cardano, then two Newton steps."""
    p = b1 - b2 * b2 / 3
    q = 2 * b2 ** 3 / 27 - b2 * b1 / 3 + b0
    disc = np.sqrt(complex(q * q / 4 + p ** 3 / 27))
    u3 = -q / 2 + disc
    if abs(-q / 2 - disc) > abs(u3):
        u3 = -q / 2 - disc
    u = u3 ** (1 / 3) if u3 != 0 else 0
    w = np.exp(2j * np.pi / 3)
    out = []
    for k in range(3):
        uk = u * w ** k
        t = uk - p / (3 * uk) if uk != 0 else 0
        out.append(t - b2 / 3)
    z = np.array(out, dtype=complex)
    for _ in range(2):
        p_ = ((z + b2) * z + b1) * z + b0
        dp = (3 * z + 2 * b2) * z + b1
        z = z - p_ / dp
    return z


def test_degree3_closed_form(orc):
    g = rng(10)
    co = crandn(g, 500, 4)
    roots, status, _, _ = orc.solve(co)
    assert np.all(status == 0)
    for i, c in enumerate(co):
        ref = _cardano(c[2] / c[3], c[1] / c[3], c[0] / c[3])
        kappa = orc.root_condition(c[None, :], ref[None, :])[0]
        assert np.all(rel_err(match(ref, roots[i]), ref) <= DEFL_BOUND * np.maximum(1.0, kappa))


def test_vieta_and_backward_error(orc):
    """The computed root set reproduces the monic coefficients (backward
    stability of the set) and every root has a small backward error."""
    co = W.gaussian(41, 2000, 6)
    roots, status, _, _ = orc.solve(co)
    assert np.all(status == 0)
    mon = co / co[:, -1:]
    for i in range(len(co)):
        expanded = np.poly(roots[i])[::-1]  # product of (z - root), lowest power first
        scale = np.abs(mon[i]).sum() * np.prod(np.maximum(1, np.abs(roots[i])))
        assert np.abs(expanded - mon[i]).max() <= 1e-12 * scale
    # elementary symmetric functions: sum and product of the roots
    assert np.allclose(roots.sum(1), -mon[:, 5], rtol=1e-10, atol=1e-10)
    assert np.allclose(np.prod(roots, 1), mon[:, 0], rtol=1e-9, atol=1e-11)
    # per-root backward error |p(z)| / sum |a_k| |z|^k
    z = roots
    p = np.zeros_like(z)
    den = np.zeros(z.shape)
    for k in range(6, -1, -1):
        p = p * z + co[:, k:k + 1]
        den = den * np.abs(z) + np.abs(co[:, k:k + 1])
    eta = np.abs(p) / den
    assert eta.max() <= 1e-12


def test_degree1_and_degenerate_inputs(orc):
    roots, status, _, _ = orc.solve(np.array([[2 + 1j, 4 - 2j]]))
    assert status[0] == 0 and roots[0, 0] == -(2 + 1j) / (4 - 2j)
    # zero leading coefficient and non-finite input -> DEGENERATE, NaN roots
    bad = np.array([[1, 2, 0], [1, np.nan, 1], [np.inf, 1, 1]], dtype=complex)
    roots, status, sweeps, _ = orc.solve(bad)
    assert np.all(status == orc.DEGENERATE) and np.all(np.isnan(roots)) and np.all(sweeps == 0)


def test_pure_rayleigh_stalls_on_littlewood_and_exceptional_shift_fixes_it(orc):
    """A real Rayleigh shift never splits a complex pair of a real matrix, so
    some {+-1, +-i} polynomials stall with the paper's shift alone; the
    exceptional Wilkinson shift (every 10 stagnant sweeps) makes all converge."""
    co = W.littlewood(2, 20000).astype(np.complex128)
    _, st_plain, _, _ = orc.solve(co, exc_period=0)
    assert (st_plain == orc.NOT_CONVERGED).sum() > 100
    _, st_exc, _, _ = orc.solve(co, exc_period=10)
    assert np.all(st_exc == 0)
    _, st_w, sw_w, _ = orc.solve(co, shift=orc.SHIFT_WILKINSON)
    assert np.all(st_w == 0)


def test_batch_is_deterministic_across_thread_counts(orc):
    co = W.gaussian(51, 3000, 6)
    r1, s1, w1, _ = orc.solve(co, threads=1)
    r4, s4, w4, _ = orc.solve(co, threads=4)
    assert np.array_equal(r1, r4) and np.array_equal(s1, s4) and np.array_equal(w1, w4)


# ----------------------------------------------------- histogram (Sec. III)

WIN1 = (-1.5, 1.5, -0.84375, 0.84375)


def test_hist_hand_computed_points(orc):
    pts = np.array([
        -1.5 + 0.84375j,                 # top-left corner -> pixel (row 0, col 0)
        0.0 + 0.0j,                      # centre -> col 960, row 540
        1.5 - 1e-12 + 0.0j,              # just inside right edge -> col 1919
        -0.84375j + 1e-12j,              # just above bottom edge -> row 1079
        1.5 + 0.0j,                      # right edge: outside (half-open)
        -0.84375j,                       # bottom edge: outside
        complex(np.nan, 0.0),            # NaN: outside
        10.0 + 0j,                       # far away: outside
    ])
    h, oow = orc.hist(pts, WIN1)
    assert oow == 4
    assert h.sum() == 4
    assert h[0, 0] == 1 and h[540, 960] == 1 and h[540, 1919] == 1 and h[1079, 960] == 1


def test_hist_matches_numpy_histogram2d(orc):
    g = rng(11)
    z = g.uniform(-1.7, 1.7, 200000) + 1j * g.uniform(-1.0, 1.0, 200000)
    xe = np.linspace(-1.5, 1.5, 1921)
    ye = np.linspace(-0.84375, 0.84375, 1081)
    # keep points well away from every bin edge, where the two edge conventions agree
    dx = np.min(np.abs(z.real[:, None] - xe[None, [0, -1]]), axis=1)
    far = (np.abs(((z.real + 1.5) * 640) - np.round((z.real + 1.5) * 640)) > 1e-6) & \
          (np.abs(((0.84375 - z.imag) * 640) - np.round((0.84375 - z.imag) * 640)) > 1e-6) & (dx > 1e-6)
    z = z[far]
    h, oow = orc.hist(z, WIN1)
    ref, _, _ = np.histogram2d(-z.imag, z.real, bins=[-ye[::-1], xe])
    assert np.array_equal(h, ref.astype(np.uint32))
    inside = (z.real >= -1.5) & (z.real < 1.5) & (z.imag > -0.84375) & (z.imag <= 0.84375)
    assert oow == int((~inside).sum())


# ------------------------------------------------ L2 approximation (Sec. II-A)

def test_gauss_legendre_matches_numpy(orc):
    for nr in (1, 2, 5, 16, 32):
        x, w = orc.gauss_legendre(nr)
        t, wt = np.polynomial.legendre.leggauss(nr)
        assert np.allclose(x, 0.5 * (t + 1), atol=2e-16, rtol=0)
        assert np.allclose(w, 0.5 * wt, atol=4e-16, rtol=0)


def test_gauss_legendre_exact_for_degree_2n_minus_1(orc):
    x, w = orc.gauss_legendre(16)
    for k in range(32):
        assert abs((w * x ** k).sum() - 1.0 / (k + 1)) <= 1e-15


def test_gram_matrix_is_diagonal_pi_over_j_plus_1(orc):
    """With the area measure, <z^j, z^k> = pi/(j+1) delta_jk on the unit disk."""
    _, G = orc.l2_approx(np.zeros((1, 512)), return_gram=True)
    assert np.allclose(G, np.diag(np.pi / np.arange(1, 8)), atol=1e-14, rtol=0)


def test_l2_reproduces_polynomials_exactly(orc):
    g = rng(12)
    a = crandn(g, 20, 7)
    w = orc.l2_nodes()
    samples = np.stack([np.polyval(ai[::-1], w) for ai in a])
    got = orc.l2_approx(samples)
    assert np.abs(got - a).max() <= 1e-13


def test_l2_worked_example_of_the_paper(orc):
    """f(z) = 1/(1 - 0.3 z), degree 6: the L2 approximation is the Taylor
    truncation (a_j = 0.3^j, the z^j are orthogonal), and its sup error on the
    unit disk, by the maximum modulus principle attained on |z| = 1, is
    0.3^7/0.7 = 3.124e-4, inside the paper's 7.3e-4; on |z| < 1e-2 it is
    below the paper's 1e-14."""
    gold = json.load(open(os.path.join(GOLDEN, "l2_worked_example.json")))
    f = lambda z: 1.0 / (1.0 - 0.3 * z)
    w = orc.l2_nodes()
    a = orc.l2_approx(f(w)[None, :])[0]
    assert np.abs(a - 0.3 ** np.arange(7)).max() <= 1e-14
    circle = np.exp(2j * np.pi * np.arange(20000) / 20000)
    sup = np.abs(f(circle) - np.polyval(a[::-1], circle)).max()
    assert sup <= gold["sup_error_unit_disk_at_most"]
    assert abs(sup - 0.3 ** 7 / 0.7) <= 1e-9
    # small disk |z| < delta: approximate g(w) = f(delta w) on the unit disk
    delta = gold["small_disk_radius"]
    ah = orc.l2_approx(f(delta * w)[None, :])[0]
    zs = delta * circle
    sup_small = np.abs(f(zs) - np.polyval(ah[::-1], zs / delta)).max()
    assert sup_small <= gold["sup_error_small_disk_at_most"]


# ---------------------------------------- implicit-differentiation adjoint

def test_adjoint_degree1_closed_form(orc):
    """z = -a0/a1: dz/da0 = -1/a1, dz/da1 = a0/a1^2 (= -z/a1)."""
    a = np.array([[1.5 - 0.5j, 0.7 + 2.0j]])
    z = -a[:, 0:1] / a[:, 1:2]
    gz = np.array([[0.3 - 1.1j]])
    g, st = orc.roots_backward(a, z, gz)
    assert st[0] == 0
    assert abs(g[0, 0] - np.conj(-1 / a[0, 1]) * gz[0, 0]) < 1e-15
    assert abs(g[0, 1] - np.conj(a[0, 0] / a[0, 1] ** 2) * gz[0, 0]) < 1e-15


def test_adjoint_of_root_sum_and_product(orc):
    """Vieta: sum z = -a_{d-1}/a_d. With L = Re(sum z) every grad_z is 1 and
    the gradient is conj(-1/a_d) on a_{d-1}, conj(a_{d-1}/a_d^2) on a_d, and
    zero elsewhere (sum_j z_j^k / p'(z_j) = 0 for k < d-1)."""
    co = W.gaussian(61, 200, 6)
    roots, _, _, _ = orc.solve(co)
    g, st = orc.roots_backward(co, roots, np.ones_like(roots))
    assert np.all(st == 0)
    scale = np.abs(g).max(axis=1, keepdims=True)
    assert np.abs(g[:, :5]).max() <= 1e-8 * scale.max()
    assert np.allclose(g[:, 5], np.conj(-1 / co[:, 6]), rtol=1e-9)
    assert np.allclose(g[:, 6], np.conj(co[:, 5] / co[:, 6] ** 2), rtol=1e-9)


def test_adjoint_matches_finite_differences_of_lapack_roots(orc):
    """Central differences (h = 1e-6) of L = sum_j w_j . z_j, with the roots
    from LAPACK (numpy) rematched to the unperturbed set."""
    g = rng(13)
    co = W.gaussian(71, 40, 6)
    z0 = np.array([np.roots(c[::-1]) for c in co])
    wts = crandn(g, *z0.shape)

    def loss(c, ref):
        z = match(ref, np.roots(c[::-1]))
        return float((wts_i.real * z.real + wts_i.imag * z.imag).sum())

    grads, st = orc.roots_backward(co, z0, wts)
    h = 1e-6
    for i in range(len(co)):
        sep = np.min(np.abs(z0[i][:, None] - z0[i][None, :]) + np.eye(6) * 1e9)
        if sep < 1e-2:
            continue
        wts_i = wts[i]
        fd = np.zeros(7, complex)
        for k in range(7):
            for unit in (1.0, 1j):
                cp = co[i].copy(); cp[k] += h * unit
                cm = co[i].copy(); cm[k] -= h * unit
                d = (loss(cp, z0[i]) - loss(cm, z0[i])) / (2 * h)
                fd[k] += d * unit
        assert np.abs(fd - grads[i]).max() <= 1e-6 * max(1.0, np.abs(grads[i]).max()), i


def test_adjoint_singular_derivative_sets_status(orc):
    a = np.array([[1.0, -2.0, 1.0]], dtype=complex)  # (z-1)^2: p'(1) = 0
    z = np.array([[1.0, 1.0]], dtype=complex)
    g, st = orc.roots_backward(a, z, np.ones_like(z))
    assert st[0] == orc.SINGULAR and np.all(g == 0)


# ------------------------------------------- paper's throughput arithmetic

def test_paper_cycle_model_consistency():
    """Sec. IV-A: n(n-1)T cycles per input at 100 MHz gives the FPGA rate of
    Table IV, and (n-1)T sweeps per polynomial give the QR/s of Table II."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_throughput.json")))
    n, T = gold["n"], gold["T"]
    cycles = T * sum(2 * m - 2 for m in range(2, n + 1))
    assert cycles == n * (n - 1) * T == 300
    rate = gold["pe_clock_hz"] / cycles
    assert abs(rate - gold["fpga_polys_per_s"]) / gold["fpga_polys_per_s"] < 0.01
    # the paper prints 16.5M for 3.33e5 * 50 = 16.65M
    assert abs(rate * (n - 1) * T - gold["fpga_equiv_qr_per_s"]) / gold["fpga_equiv_qr_per_s"] < 0.02


# ------------------------------------------- helpers of the full pipeline

def test_affine_map_is_centre_plus_radius_times_w(orc):
    g = rng(21)
    w = crandn(g, 50, 6)
    c = crandn(g, 50)
    got = orc.affine(w, c, 0.25)
    assert np.array_equal(got, c[:, None] + 0.25 * w)


def test_tiled_histogram_keeps_only_roots_in_their_own_tile(orc):
    """A 4 x 2 tile grid over [0,4) x (0,2]: tile t = row * 4 + col, rows from
    the top. Hand-placed roots: in own tile, in a neighbour, outside."""
    win = (0.0, 4.0, 0.0, 2.0)
    roots = np.array([[0.5 + 1.5j, 1.5 + 1.5j],     # poly 0 (tile 0): kept, dropped (tile 1)
                      [3.5 + 0.5j, 3.9 + 0.1j],     # poly 1 (tile 7): both kept
                      [9.0 + 0.0j, 2.5 + 0.5j]])    # poly 2 (tile 6): outside, kept
    tiles = np.array([0, 7, 6])
    h, oow, dropped = orc.hist_tiled(roots, tiles, 4, 2, win, W=8, H=4)
    assert dropped == 2 and oow == 0 and h.sum() == 4
    # pixels are 0.5 x 0.5: 0.5+1.5i -> row 1, col 1; 3.5+0.5i and 3.9+0.1i -> row 3, col 7;
    # 2.5+0.5i -> row 3, col 5
    assert h[1, 1] == 1 and h[3, 7] == 2 and h[3, 5] == 1


def test_root_condition_closed_form(orc):
    """p = (z-1)(z-2) = 2 - 3z + z^2: at z = 1, sum |a_k| |z|^k = 6 and
    |p'(1)| = 1, so kappa = 6; at z = 2, (2 + 6 + 4) / (2 * 1) = 6."""
    k = orc.root_condition(np.array([[2, -3, 1]], complex), np.array([[1, 2]], complex))
    assert np.allclose(k, [[6.0, 6.0]], rtol=1e-15)


# ------------------------------------------- Alg. 2's fixed schedule

def test_fixed_schedule_converges_to_the_roots_with_enough_sweeps(orc):
    """With T = 30 sweeps per eigenvalue and the Wilkinson shift, Alg. 2's
    fixed schedule reaches the same roots as LAPACK."""
    co = W.gaussian(81, 300, 6)
    roots, status = orc.solve_fixed(co, T=30, shift=orc.SHIFT_WILKINSON)
    assert np.all(status == 0)
    ref = np.array([np.roots(c[::-1]) for c in co])
    kappa = orc.root_condition(co, ref)
    err = matched_errors(roots, ref)
    assert np.all(err <= DEFL_BOUND * np.maximum(1.0, kappa))


def test_fixed_schedule_with_paper_settings_mostly_converges(orc):
    """T = 10 and the paper's Rayleigh shift (Sec. IV settings): about 90 % of
    unit-disk polynomials have every root right to 1e-6, and doubling T
    brings nearly all of them in; the fixed schedule has no test that would
    stop a level early or keep it going."""
    co, true_roots = W.unit_disk_roots(1, 2000)
    roots, status = orc.solve_fixed(co, T=10)
    ok10 = (matched_errors(roots, true_roots).max(axis=1) < 1e-6).mean()
    roots, status = orc.solve_fixed(co, T=20)
    ok20 = (matched_errors(roots, true_roots).max(axis=1) < 1e-6).mean()
    assert 0.85 < ok10 < 0.95 and ok20 > 0.995


# --------------------------------- soft root density (differentiation workload)

SPLAT_WIN = (-2.0, 2.0, -1.125, 1.125)  # 256 x 144 pixels of 1/64


def test_splat_mass_averaged_over_subpixel_offsets_is_the_integral(orc):
    """Averaged over a 16 x 16 grid of sub-pixel positions, the image mass of
    one root equals the integral of the truncated bump over the plane
    (Poisson summation): pi sigma^2 (2 - 11 e^{-9/2}) for the cut at 3 sigma."""
    px = 4.0 / 256
    tot = [orc.splat(np.array([(a + 0.5) / 16 * px + 1j * (b + 0.5) / 16 * px]), SPLAT_WIN).sum()
           for a in range(16) for b in range(16)]
    exact = math.pi * 1.5 ** 2 * (2.0 - 11.0 * math.exp(-4.5))
    assert abs(np.mean(tot) / exact - 1.0) <= 3e-6


def test_splat_of_a_root_at_a_pixel_centre_is_symmetric_and_peaks_there(orc):
    """A root at the centre of pixel (iy, ix) (dyadic coordinates, exact in
    pixel units): the image is symmetric under x and y reflection about that
    pixel, peaks at 1 - e^{-9/2} there, and that pixel is the one the
    histogram's binning (row 0 at ymax) assigns to the root."""
    ix, iy = 100, 40
    z = complex(-2.0 + (ix + 0.5) / 64, 1.125 - (iy + 0.5) / 64)
    img = orc.splat(np.array([z]), SPLAT_WIN)
    assert np.unravel_index(np.argmax(img), img.shape) == (iy, ix)
    assert img[iy, ix] == 1.0 - math.exp(-4.5)
    box = img[iy - 6:iy + 7, ix - 6:ix + 7]
    assert np.array_equal(box, box[::-1, :]) and np.array_equal(box, box[:, ::-1])
    assert np.array_equal(box, box.T)
    rest = img.copy()
    rest[iy - 6:iy + 7, ix - 6:ix + 7] = 0.0
    assert not rest.any()  # nothing beyond 6 pixels
    h, _ = orc.hist(np.array([z]), SPLAT_WIN, 256, 144)
    assert h[iy, ix] == 1


def test_splat_moves_with_the_root(orc):
    """Shifting a root by exactly one pixel (dyadic steps) shifts its image by
    one pixel, bit for bit; a NaN root or one 10 pixels outside adds nothing."""
    z = complex(0.25 + 3.0 / 1024, -0.5 + 5.0 / 1024)
    a = orc.splat(np.array([z]), SPLAT_WIN)
    b = orc.splat(np.array([z + 1.0 / 64]), SPLAT_WIN)
    c = orc.splat(np.array([z - 1j / 64]), SPLAT_WIN)
    assert np.array_equal(a[:, :-1], b[:, 1:]) and np.array_equal(a[:-1, :], c[1:, :])
    far = orc.splat(np.array([complex(np.nan, 0.0), 2.0 + 10.0 / 64 + 0j]), SPLAT_WIN)
    assert not far.any()


def test_splat_gradient_is_the_derivative_of_the_image(orc):
    """dL/dRe z, dL/dIm z of L = sum G * img against central differences of
    the oracle's own image (h = 1e-7), for 50 roots and a random G."""
    g = rng(91)
    z = g.uniform(-1.9, 1.9, 50) + 1j * g.uniform(-1.0, 1.0, 50)
    G = g.standard_normal((144, 256))
    grad = orc.splat_grad(z, G, SPLAT_WIN, scale=0.5)
    h = 1e-7
    for j in range(z.size):
        fd = 0j
        for unit in (1.0, 1j):
            lp = (G * orc.splat(np.array([z[j] + h * unit]), SPLAT_WIN, scale=0.5)).sum()
            lm = (G * orc.splat(np.array([z[j] - h * unit]), SPLAT_WIN, scale=0.5)).sum()
            fd += unit * (lp - lm) / (2 * h)
        assert abs(fd - grad[j]) <= 1e-6 * max(1.0, abs(grad[j])), (j, fd, grad[j])
