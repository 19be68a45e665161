"""GPU parity of the L2 approximation and of the full pipeline (tiles -> L2 ->
roots -> clip -> histogram) against the oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2507_02164_gb300 import api, workloads as WL
from tests.gpu_common import hist_np, require_gpu, roots_poly_major

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def test_l2_matches_oracle_on_random_samples(dev, orc):
    g = np.random.default_rng(2)
    n = 3000 + 7
    s = g.standard_normal((n, 512)) + 1j * g.standard_normal((n, 512))
    got = api.l2_approx(torch.from_numpy(s).to(dev), 16, 32, 6)
    torch.cuda.synchronize()
    ref = orc.l2_approx(s)
    assert np.abs(got.cpu().numpy().T - ref).max() <= 1e-13


def test_l2_worked_example(dev):
    """f = 1/(1 - 0.3 w): the L2 coefficients are 0.3^j (Sec. II-A example)."""
    w = api.l2_sample_points(16, 32, dev)
    s = (1.0 / (1.0 - 0.3 * w))[None, :].contiguous()
    a = api.l2_approx(s, 16, 32, 6).cpu().numpy()[:, 0]
    assert np.abs(a - 0.3 ** np.arange(7)).max() <= 1e-14


# (16, 6) runs the build specialised for the pipeline's node count and
# degree; every other pair the build with runtime bounds
@pytest.mark.parametrize("degree,nr", [(0, 1), (3, 8), (12, 32), (6, 8), (5, 16), (6, 16)])
@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_l2_degree_and_radial_order_range(dev, orc, degree, nr, precision):
    g = np.random.default_rng(degree)
    s = g.standard_normal((100, nr * 32)) + 1j * g.standard_normal((100, nr * 32))
    got = api.l2_approx(torch.from_numpy(s).to(dev), nr, 32, degree, precision=precision).cpu().numpy().T
    ref = orc.l2_approx(s, nr=nr, nt=32, degree=degree)
    assert np.abs(got - ref).max() <= 1e-12


def test_full_pipeline_block_of_tiles(dev, orc):
    """f(z) = sin(z^3) + 0.5 z on the 480 x 270 tile grid, a block of rows:
    L2 on each sub-disk, mixed roots, clip to the own tile, histogram."""
    win = (-4.0, 4.0, -2.25, 2.25)
    centres, rho, _, _ = WL.tiles(*win, 480, 270)
    rows = slice(100 * 480, 140 * 480)  # 40 full tile rows through the middle
    c = centres[rows]
    tile_idx = np.arange(100 * 480, 140 * 480, dtype=np.int64)
    w = orc.l2_nodes(16, 32)
    samples = WL.f_sin_cube(c[:, None] + rho * w[None, :])
    # GPU: L2 -> fused mixed roots + clip + histogram
    s_t = torch.from_numpy(np.ascontiguousarray(samples)).to(dev)
    coeffs = api.l2_approx(s_t, 16, 32, 6)
    hist = api.new_hist(1920, 1080, dev)
    roots = torch.empty((6, c.size), dtype=torch.complex128, device=dev)
    stats = api.new_stats(dev)
    clip = api.make_clip(torch.from_numpy(c).to(dev), rho, 480, 270, api.Window(*win),
                         torch.from_numpy(tile_idx).to(dev))
    api.roots_density(coeffs, api.Window(*win), hist, mode="mixed", clip=clip, roots=roots, stats=stats)
    torch.cuda.synchronize()
    h_gpu = hist_np(hist)
    r_gpu = roots_poly_major(roots)
    # the oracle's clip + binning of the GPU's roots reproduces the GPU histogram exactly
    z_gpu = orc.affine(r_gpu, c, rho)
    h_ref, oow, dropped = orc.hist_tiled(z_gpu, tile_idx, 480, 270, win)
    assert np.array_equal(h_gpu, h_ref)
    st = api.stats_dict(stats)
    assert st["clipped"] == dropped and st["binned"] == int(h_ref.sum())
    # the oracle's own pipeline gives the same kept roots
    co_ref = orc.l2_approx(samples)
    r_ref, _, _, _ = orc.solve(co_ref)
    h_or, _, _ = orc.hist_tiled(orc.affine(r_ref, c, rho), tile_idx, 480, 270, win)
    assert abs(int(h_or.sum()) - int(h_gpu.sum())) <= 2
    # kept roots are zeros of f: one FP64 Newton step on f moves them by < 1e-6
    ys, xs = np.nonzero(h_gpu)
    assert h_gpu.sum() >= 20
    kept = z_gpu.reshape(-1)
    fz = WL.f_sin_cube(kept)
    fp = 3 * kept ** 2 * np.cos(kept ** 3) + 0.5
    keep_mask = np.zeros(kept.size, bool)
    t = np.floor((kept.real + 4.0) * 60).astype(np.int64) + 480 * np.floor((2.25 - kept.imag) * 60).astype(np.int64)
    keep_mask = t == np.repeat(tile_idx, 6)
    step = np.abs(fz / fp)[keep_mask]
    assert np.all(step < 1e-6), step.max()


def test_full_pipeline_all_tiles(dev, orc):
    """All 129,600 sub-disks of the 480 x 270 grid, as bench.py times them:
    the fused histogram equals the oracle's clip + binning of the GPU roots
    bit for bit, the L2 coefficients of a sample of 2,000 sub-disks match the
    oracle's, and every kept root is a zero of f (one Newton step on f moves
    it by less than 1e-6)."""
    win = (-4.0, 4.0, -2.25, 2.25)
    centres, rho, _, _ = WL.tiles(*win, 480, 270)
    c = torch.from_numpy(centres).to(dev)
    w = api.l2_sample_points(16, 32, dev)
    samples = WL.f_sin_cube(c[:, None] + rho * w[None, :]).contiguous()
    coeffs = api.l2_approx(samples, 16, 32, 6)
    hist = api.new_hist(1920, 1080, dev)
    roots = torch.empty((6, c.numel()), dtype=torch.complex128, device=dev)
    stats = api.new_stats(dev)
    clip = api.make_clip(c, rho, 480, 270, api.Window(*win))
    api.roots_density(coeffs, api.Window(*win), hist, mode="mixed", clip=clip, roots=roots, stats=stats)
    torch.cuda.synchronize()
    z = orc.affine(roots_poly_major(roots), centres, rho)
    h_ref, oow, dropped = orc.hist_tiled(z, np.arange(c.numel()), 480, 270, win)
    assert np.array_equal(hist_np(hist), h_ref)
    st = api.stats_dict(stats)
    assert st["clipped"] == dropped and st["binned"] == int(h_ref.sum())
    idx = np.linspace(0, c.numel() - 1, 2000).astype(np.int64)
    ref = orc.l2_approx(samples.cpu().numpy()[idx])
    # |sin(z^3)| reaches ~1e41 at the window corners: compare relative to each
    # sub-disk's largest coefficient
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert (np.abs(coeffs.cpu().numpy().T[idx] - ref) / scale).max() <= 1e-13
    zz = z.reshape(-1)
    tx = np.floor((zz.real + 4.0) * 60).astype(np.int64)
    ty = np.floor((2.25 - zz.imag) * 60).astype(np.int64)
    own = (tx == np.repeat(np.arange(c.numel()), 6) % 480) & (ty == np.repeat(np.arange(c.numel()), 6) // 480)
    k = zz[own & np.isfinite(zz)]
    assert k.size == st["binned"]
    step = np.abs(WL.f_sin_cube(k) / (3 * k ** 2 * np.cos(k ** 3) + 0.5))
    assert np.all(step < 1e-6), step.max()


# ---------------------------------------------- double-float L2 variant

def test_l2_double_float_matches_oracle(dev, orc):
    """RD_L2_DF on random samples of widely varying scale (each sub-disk
    scaled by up to 2^+-120): within 1e-13 of the oracle relative to each
    sub-disk's largest coefficient; the worked example within 1e-13."""
    g = np.random.default_rng(4)
    n = 3000 + 7
    s = g.standard_normal((n, 512)) + 1j * g.standard_normal((n, 512))
    s *= 2.0 ** g.integers(-120, 120, size=(n, 1))
    got = api.l2_approx(torch.from_numpy(s).to(dev), 16, 32, 6, precision="df").cpu().numpy().T
    ref = orc.l2_approx(s)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert (np.abs(got - ref) / scale).max() <= 1e-13
    w = api.l2_sample_points(16, 32, dev)
    a = api.l2_approx((1.0 / (1.0 - 0.3 * w))[None, :].contiguous(), 16, 32, 6, precision="df").cpu().numpy()[:, 0]
    assert np.abs(a - 0.3 ** np.arange(7)).max() <= 1e-13


def test_l2_double_float_on_the_full_tile_grid(dev, orc):
    win = (-4.0, 4.0, -2.25, 2.25)
    centres, rho, _, _ = WL.tiles(*win, 480, 270)
    c = torch.from_numpy(centres).to(dev)
    w = api.l2_sample_points(16, 32, dev)
    samples = WL.f_sin_cube(c[:, None] + rho * w[None, :]).contiguous()
    df = api.l2_approx(samples, 16, 32, 6, precision="df").cpu().numpy().T
    fp = api.l2_approx(samples, 16, 32, 6, precision="fp64").cpu().numpy().T
    scale = np.abs(fp).max(axis=1, keepdims=True)
    assert (np.abs(df - fp) / scale).max() <= 1e-13
