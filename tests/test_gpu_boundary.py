"""GPU parity of the boundary calls that act on roots obtained elsewhere:
standalone binning with a status mask and the sub-disk tile clip (Sec. II
subregions, Sec. III roots to pixels), the packed uneven-degree adjoint, the
affine map of rd_l2_approx and the ALU throughput probe."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_2507_02164_gb300 import _native as N
from paper_2507_02164_gb300 import api, workloads as WL
from tests.gpu_common import hist_np, require_gpu, roots_poly_major, to_soa

pytestmark = pytest.mark.gpu

WIN1 = api.Window(-1.5, 1.5, -0.84375, 0.84375)


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def test_status_mask_bins_only_ok_polynomials(dev, orc):
    """Roots [d, n] with a status per polynomial: the image equals the
    oracle's binning of the roots of the OK polynomials alone, and every other
    root is counted as dropped."""
    n, d = 20000 + 11, 6
    co, _ = WL.unit_disk_roots(1, n)
    roots, _, _, _ = orc.solve(co)
    rng = np.random.default_rng(5)
    status = rng.choice(np.array([0, 1, 2, 3], np.uint8), size=n, p=[0.85, 0.05, 0.05, 0.05])
    r_t = to_soa(roots, dev)
    s_t = torch.from_numpy(status).to(dev)
    hist = api.new_hist(1920, 1080, dev)
    stats = api.new_stats(dev)
    api.density_accumulate(r_t, WIN1, hist, status=s_t, stats=stats)
    torch.cuda.synchronize()
    h_ref, oow = orc.hist(roots[status == 0], WIN1.tuple(), 1920, 1080)
    assert np.array_equal(hist_np(hist), h_ref)
    st = api.stats_dict(stats)
    assert st["clipped"] == d * int((status != 0).sum())
    assert st["binned"] == int(h_ref.sum()) and st["out_of_window"] == oow
    # without the mask every root counts
    h2 = api.new_hist(1920, 1080, dev)
    api.density_accumulate(r_t, WIN1, h2)
    torch.cuda.synchronize()
    assert np.array_equal(hist_np(h2), orc.hist(roots, WIN1.tuple(), 1920, 1080)[0])


@pytest.mark.parametrize("explicit_tiles", [False, True])
def test_standalone_tile_clip_matches_oracle_bit_for_bit(dev, orc, explicit_tiles):
    """The sub-disk pipeline split in two calls: roots solved without binning,
    then binned with the own-tile clip by rd_density_accumulate. The image
    equals the oracle's map + clip + binning of the same roots bit for bit,
    and the fused solve's image (clip inside the solve) as well. With
    tile_index the polynomials are a shuffled subset of the grid's tiles."""
    win = (-4.0, 4.0, -2.25, 2.25)
    nx, ny = 480, 270
    centres, rho, _, _ = WL.tiles(*win, nx, ny)
    tiles_idx = np.arange(centres.size, dtype=np.int64)
    if explicit_tiles:
        tiles_idx = np.random.default_rng(9).permutation(centres.size)[:50000].astype(np.int64)
    cen = centres[tiles_idx]
    c_t = torch.from_numpy(cen).to(dev)
    w = api.l2_sample_points(16, 32, dev)
    samples = WL.f_sin_cube(c_t[:, None] + rho * w[None, :]).contiguous()
    clip = N.Clip()
    coeffs = api.l2_approx(samples, 16, 32, 6, centres=c_t, radius=rho, clip=clip)
    assert clip.centres == c_t.data_ptr() and clip.radius == rho
    clip.nx, clip.ny, clip.tiles = nx, ny, api.Window(*win).c()
    t_t = torch.from_numpy(tiles_idx).to(dev) if explicit_tiles else None
    clip.tile_index = t_t.data_ptr() if t_t is not None else None
    roots, status = api.roots_batched(coeffs, mode="mixed")
    hist = api.new_hist(1920, 1080, dev)
    stats = api.new_stats(dev)
    api.density_accumulate(roots, api.Window(*win), hist, clip=clip, stats=stats)
    fused = api.new_hist(1920, 1080, dev)
    fstats = api.new_stats(dev)
    api.roots_density(coeffs, api.Window(*win), fused, mode="mixed", clip=clip, stats=fstats)
    torch.cuda.synchronize()
    z = orc.affine(roots_poly_major(roots), cen, rho)
    h_ref, oow, dropped = orc.hist_tiled(z, tiles_idx, nx, ny, win)
    assert np.array_equal(hist_np(hist), h_ref)
    assert np.array_equal(hist_np(fused), h_ref)
    st, fs = api.stats_dict(stats), api.stats_dict(fstats)
    assert st["clipped"] == dropped == fs["clipped"]
    assert st["binned"] == int(h_ref.sum()) == fs["binned"] and st["out_of_window"] == oow
    assert h_ref.sum() > 0


def _packed(seed, n, dtype):
    packed, deg, off = WL.uneven_gaussian(seed, n, dtype=dtype)
    return packed, deg, off


@pytest.mark.parametrize("dtype,rtol", [(np.complex128, 1e-12), (np.complex64, 1e-4)])
def test_packed_adjoint_matches_oracle_per_degree(dev, orc, dtype, rtol):
    """rd_roots_backward_uneven on a packed batch of degrees 2..12 equals the
    oracle's adjoint of every degree bin (roots from the oracle, random
    gradients)."""
    n = 6000 + 7
    packed, deg, off = _packed(3, n, dtype)
    pk = packed.astype(np.complex128)
    n_roots = packed.size - n
    roots = np.zeros(n_roots, np.complex128)
    rng = np.random.default_rng(4)
    gz = rng.standard_normal(n_roots) + 1j * rng.standard_normal(n_roots)
    ref_grad = np.zeros(packed.size, np.complex128)
    ref_status = np.zeros(n, np.uint8)
    for d in np.unique(deg):
        idx = np.nonzero(deg == d)[0]
        rows = np.stack([pk[off[i]:off[i + 1]] for i in idx])
        z, _, _, _ = orc.solve(rows)
        g = np.stack([gz[off[i] - i: off[i] - i + d] for i in idx])
        gr, gs = orc.roots_backward(rows, z, g)
        for k, i in enumerate(idx):
            roots[off[i] - i: off[i] - i + d] = z[k]
            ref_grad[off[i]:off[i + 1]] = gr[k]
        ref_status[idx] = gs
    tdt = torch.complex128 if dtype == np.complex128 else torch.complex64
    status = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    got = api.roots_backward_uneven(torch.from_numpy(packed).to(dev), torch.from_numpy(deg).to(dev),
                                    torch.from_numpy(off).to(dev), torch.from_numpy(roots).to(dev),
                                    torch.from_numpy(gz).to(dev), status=status)
    torch.cuda.synchronize()
    g = got.cpu().numpy().astype(np.complex128)
    assert np.array_equal(status.cpu().numpy(), ref_status)
    for d in np.unique(deg):
        idx = np.nonzero(deg == d)[0]
        a = np.stack([g[off[i]:off[i + 1]] for i in idx])
        b = np.stack([ref_grad[off[i]:off[i + 1]] for i in idx])
        scale = np.maximum(np.abs(b).max(axis=1, keepdims=True), 1e-300)
        assert (np.abs(a - b) / scale).max() <= rtol, d
    assert got.dtype == tdt


def test_packed_adjoint_of_one_degree_equals_the_uniform_adjoint_bit_for_bit(dev, orc):
    """A packed batch whose polynomials all have degree 6 gives the uniform
    kernel's gradients bit for bit (same operations in the same order)."""
    n, d = 3000, 6
    co = WL.gaussian(4, n, d)
    z, _, _, _ = orc.solve(co)
    rng = np.random.default_rng(8)
    gz = rng.standard_normal(z.shape) + 1j * rng.standard_normal(z.shape)
    uni = api.roots_backward(to_soa(co, dev), to_soa(z, dev), to_soa(gz, dev)).cpu().numpy().T
    off = np.arange(n + 1, dtype=np.int64) * (d + 1)
    got = api.roots_backward_uneven(torch.from_numpy(co.reshape(-1)).to(dev),
                                    torch.full((n,), d, dtype=torch.uint8, device=dev), torch.from_numpy(off).to(dev),
                                    torch.from_numpy(z.reshape(-1)).to(dev), torch.from_numpy(gz.reshape(-1)).to(dev))
    g = got.cpu().numpy().reshape(n, d + 1)
    assert np.array_equal(g.view(np.int64), np.ascontiguousarray(uni).view(np.int64))


def test_packed_adjoint_malformed_offsets_write_nothing_outside(dev):
    """Inconsistent polynomials are DEGENERATE with nothing written; a
    consistent one of degree 0 gets a zero gradient; guards stay intact."""
    deg = np.array([6, 0, 6, 3, 6], np.uint8)
    off = np.array([0, 7, 8, 3, 20, 27], np.int64)  # poly 2 runs backwards, poly 3 [3, 20) is 17 long
    n, n_coeffs = 5, 27
    rng = np.random.default_rng(0)
    coeffs = rng.standard_normal(n_coeffs) + 1j * rng.standard_normal(n_coeffs)
    roots = rng.standard_normal(n_coeffs - n) + 1j * rng.standard_normal(n_coeffs - n)
    grad_buf = torch.full((n_coeffs + 64,), complex(5.0, 5.0), dtype=torch.complex128, device=dev)
    status = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    api.roots_backward_uneven(torch.from_numpy(coeffs).to(dev), torch.from_numpy(deg).to(dev),
                              torch.from_numpy(off).to(dev), torch.from_numpy(roots).to(dev),
                              torch.from_numpy(roots).to(dev), grad_coeffs=grad_buf[:n_coeffs], status=status)
    torch.cuda.synchronize()
    s = status.cpu().numpy()
    g = grad_buf.cpu().numpy()
    assert s[1] == 3 and s[2] == 3 and s[3] == 3
    assert s[0] in (0, 2) and s[4] in (0, 2)
    assert g[7] == 0  # degree 0: zero gradient for its one coefficient
    assert np.all(g[n_coeffs:] == complex(5.0, 5.0))
    assert np.all(g[8:20] == complex(5.0, 5.0))  # nothing of polynomials 2, 3 written


def test_alu_probe_measures_a_plausible_rate(dev):
    """The FFMA / DFMA probe runs, reports its flops, and measures a rate
    between 20 % and 130 % of the nominal peak of 152 SMs at 2.07 GHz
    (FP32: 128 FMA lanes per SM; FP64: 2 per SM per clock)."""
    nominal = {"fp32": 152 * 128 * 2 * 2.07e9, "fp64": 152 * 2 * 2 * 2.07e9}
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    for kind, iters in (("fp32", 1000), ("fp64", 40)):
        api.alu_peak(kind, iters, sink=sink)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        flops = api.alu_peak(kind, iters, sink=sink)
        e1.record()
        torch.cuda.synchronize()
        rate = flops / (e0.elapsed_time(e1) * 1e-3)
        assert flops == 4 * N.load().rd_device_sm_count() * 256 * iters * (256 if kind == "fp32" else 128) * 2
        assert 0.2 * nominal[kind] <= rate <= 1.3 * nominal[kind], (kind, rate / nominal[kind])
    assert sink.item() == 0.0
