"""GPU parity of the uneven-degree path (degree bin & pack + persistent
per-degree solvers) against the FP64 CPU oracle, and its CUDA-graph capture."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2507_02164_gb300 import api, workloads as WL
from tests.gpu_common import check_rejected, compare_roots, hist_np, require_gpu

pytestmark = pytest.mark.gpu

WIN3 = api.Window(-3.0, 3.0, -1.6875, 1.6875)
W, H = 1920, 1080


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _split(packed, deg, off):
    """Per-degree lists of (poly indices, coefficient rows) of a packed batch."""
    out = {}
    for d in np.unique(deg):
        idx = np.nonzero(deg == d)[0]
        rows = np.stack([packed[off[i]:off[i + 1]] for i in idx])
        out[int(d)] = (idx, rows)
    return out


def _check_against_oracle(orc, packed, deg, off, roots, status, tol, kcap, max_rejected=2e-3):
    """Compare each degree bin's GPU roots with the oracle; return the OK mask."""
    ok = status == 0
    assert np.all((status == 0) | (status == 2)), np.bincount(status, minlength=4)
    assert (status == 2).mean() <= max_rejected
    for d, (idx, rows) in _split(packed, deg, off).items():
        r_gpu = np.stack([roots[off[i] - i: off[i] - i + d] for i in idx])
        ref, ref_st, _, _ = orc.solve(rows)
        check_rejected(rows, status[idx], ref, orc)
        good = ok[idx] & (ref_st == 0)
        assert good.mean() > 0.99, (d, good.mean())
        compare_roots(r_gpu[good], ref[good], rows[good], orc, tol, kcap)
    return ok


@pytest.mark.parametrize("mode,dtype", [("mixed", torch.complex64), ("plain", torch.complex128)])
def test_uneven_batch_matches_oracle(dev, orc, mode, dtype):
    n = 20000 + 13
    packed, deg, off = WL.uneven_gaussian(3, n, dtype=np.complex64 if dtype == torch.complex64 else np.complex128)
    c_t = torch.from_numpy(packed).to(dev)
    d_t = torch.from_numpy(deg).to(dev)
    o_t = torch.from_numpy(off).to(dev)
    ws = api.new_uneven_workspace(n, packed.size, dtype, dev)
    hist = api.new_hist(W, H, dev)
    stats = api.new_stats(dev)
    roots, status = api.roots_uneven(c_t, d_t, o_t, ws, mode=mode, window=WIN3, hist=hist, stats=stats)
    torch.cuda.synchronize()
    r = roots.cpu().numpy()
    s = status.cpu().numpy()
    tol, kcap = (1e-9, 1e3) if mode == "mixed" else (1e-11, 100.0)
    _check_against_oracle(orc, packed.astype(np.complex128), deg, off, r, s, tol, kcap)
    h_ref, oow = orc.hist(r, WIN3.tuple(), W, H)
    assert np.array_equal(hist_np(hist), h_ref)
    st = api.stats_dict(stats)
    assert st["polys"] == n and st["binned"] == int(h_ref.sum()) and st["out_of_window"] == oow
    assert st["status_ok"] == int((s == 0).sum())


@pytest.mark.parametrize("mode,dtype,polish", [("mixed", torch.complex128, "fp64"), ("plain", torch.complex64, "fp64"),
                                               ("mixed", torch.complex64, "df")])
def test_uneven_degrees_one_to_twelve(dev, orc, mode, dtype, polish):
    """Every degree 1..12 in one packed batch (degree 1 included, which the
    benchmark's 2..12 mix leaves out), in the storage / precision pairs the
    other parity test does not cover, and the compensated polish."""
    g = np.random.default_rng(29)
    n = 6000 + 7
    deg = g.integers(1, 13, n).astype(np.uint8)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg.astype(np.int64) + 1, out=off[1:])
    npd = np.complex64 if dtype == torch.complex64 else np.complex128
    packed = (g.standard_normal(int(off[-1])) + 1j * g.standard_normal(int(off[-1]))).astype(npd)
    c_t = torch.from_numpy(packed).to(dev)
    ws = api.new_uneven_workspace(n, packed.size, dtype, dev)
    p = api.params(mode, polish_mode=polish) if mode == "mixed" else api.params(mode)
    roots, status = api.roots_uneven(c_t, torch.from_numpy(deg).to(dev), torch.from_numpy(off).to(dev), ws,
                                     mode=mode, params_=p)
    torch.cuda.synchronize()
    tol, kcap = (1e-9, 1e3) if mode == "mixed" else (1e-11, 100.0)
    _check_against_oracle(orc, packed.astype(np.complex128), deg, off, roots.cpu().numpy(), status.cpu().numpy(),
                          tol, kcap)
    assert set(np.unique(deg).tolist()) == set(range(1, 13))


def test_invalid_degrees_and_offsets(dev, orc):
    packed, deg, off = WL.uneven_gaussian(3, 200)
    deg = deg.copy()
    off = off.copy()
    # polynomial 5: degree 0 with one coefficient (consistent offsets, unsolvable)
    # polynomial 9: degree field disagrees with its offsets (inconsistent)
    # rebuild the packed arrays with polynomial 5 reduced to one coefficient
    rows = [packed[off[i]:off[i + 1]] for i in range(200)]
    rows[5] = rows[5][:1]
    deg[5] = 0
    off = np.zeros(201, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    packed = np.concatenate(rows).astype(np.complex64)
    deg[9] = deg[9] + 1
    ws = api.new_uneven_workspace(200, packed.size, torch.complex64, dev)
    roots = torch.full((packed.size - 200,), 7.0 + 7.0j, dtype=torch.complex128, device=dev)
    roots_out, status = api.roots_uneven(torch.from_numpy(packed).to(dev), torch.from_numpy(deg).to(dev),
                                         torch.from_numpy(off).to(dev), ws, mode="mixed", roots=roots)
    torch.cuda.synchronize()
    s = status.cpu().numpy()
    r = roots_out.cpu().numpy()
    assert s[5] == 3 and s[9] == 3
    others = np.setdiff1d(np.arange(200), [5, 9])
    assert np.all(s[others] != 3)
    # polynomial 9's root slots are left untouched (its offsets are not trusted)
    d9 = int(deg[9]) - 1
    assert np.all(r[off[9] - 9: off[9] - 9 + d9] == 7.0 + 7.0j)


def test_workspace_too_small_is_rejected(dev):
    packed, deg, off = WL.uneven_gaussian(3, 100)
    ws = torch.empty(1024, dtype=torch.uint8, device=dev)
    with pytest.raises(api.N.RootDensityError):
        api.roots_uneven(torch.from_numpy(packed).to(dev), torch.from_numpy(deg).to(dev),
                         torch.from_numpy(off).to(dev), ws)


def test_uneven_call_captures_into_a_cuda_graph(dev):
    n = 50000
    packed, deg, off = WL.uneven_gaussian_torch(3, 0, n, dev)
    ws = api.new_uneven_workspace(n, packed.numel(), torch.complex64, dev)
    hist = api.new_hist(W, H, dev)
    roots = torch.empty(packed.numel() - n, dtype=torch.complex128, device=dev)
    status = torch.empty(n, dtype=torch.uint8, device=dev)
    api.roots_uneven(packed, deg, off, ws, window=WIN3, hist=hist, roots=roots, status=status)
    torch.cuda.synchronize()
    eager_hist = hist.clone()
    eager_roots = roots.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            api.hist_clear(hist)
            api.roots_uneven(packed, deg, off, ws, window=WIN3, hist=hist, roots=roots, status=status)
    torch.cuda.current_stream().wait_stream(s)
    roots.zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(hist, eager_hist)
    assert torch.equal(roots, eager_roots)


def test_full_size_batch_sampled(dev, orc):
    """The 2^24-polynomial uneven batch in the benchmark's configuration:
    every counter adds up, and a sample of 4096 polynomials spread over the
    batch (their stored coefficients read back from the device) matches the
    oracle."""
    n = 1 << 24
    packed, deg, off = WL.uneven_gaussian_torch(3, 0, n, dev)
    ws = api.new_uneven_workspace(n, packed.numel(), torch.complex64, dev)
    hist = api.new_hist(W, H, dev)
    stats = api.new_stats(dev)
    roots, status = api.roots_uneven(packed, deg, off, ws, window=WIN3, hist=hist, stats=stats)
    torch.cuda.synchronize()
    st = api.stats_dict(stats)
    total_roots = packed.numel() - n
    assert st["polys"] == n
    assert st["binned"] + st["out_of_window"] == total_roots
    assert int(hist_np(hist).sum(dtype=np.int64)) == st["binned"]
    s = status.cpu().numpy()
    assert (s == 0).mean() > 0.999 and np.all((s == 0) | (s == 2))
    sample = np.linspace(0, n - 1, 4096).astype(np.int64)
    off_h = off.cpu().numpy()
    deg_h = deg.cpu().numpy()
    pk = packed.cpu().numpy().astype(np.complex128)
    r = roots.cpu().numpy()
    for d in range(2, 13):
        idx = sample[deg_h[sample] == d]
        if idx.size == 0:
            continue
        rows = np.stack([pk[off_h[i]:off_h[i + 1]] for i in idx])
        r_gpu = np.stack([r[off_h[i] - i: off_h[i] - i + d] for i in idx])
        ref, ref_st, _, _ = orc.solve(rows)
        check_rejected(rows, s[idx], ref, orc)
        good = (s[idx] == 0) & (ref_st == 0)
        compare_roots(r_gpu[good], ref[good], rows[good], orc, 1e-9, 1e3)


def test_uneven_inputs_in_page_locked_host_memory(dev):
    """The count and pack kernels read coefficients, degrees and offsets from
    page-locked host memory (zero copy): same roots, status and histogram as
    from device memory."""
    n = 30000 + 5
    packed, deg, off = WL.uneven_gaussian(7, n)
    c_d, d_d, o_d = (torch.from_numpy(x).to(dev) for x in (packed, deg, off))
    c_h, d_h, o_h = (torch.from_numpy(x).pin_memory() for x in (packed, deg, off))
    ws = api.new_uneven_workspace(n, packed.size, torch.complex64, dev)
    out = []
    for c, d, o in ((c_d, d_d, o_d), (c_h, d_h, o_h)):
        hist = api.new_hist(W, H, dev)
        r, s = api.roots_uneven(c, d, o, ws, mode="mixed", window=WIN3, hist=hist)
        torch.cuda.synchronize()
        out.append((r.cpu(), s.cpu(), hist.cpu()))
    assert all(torch.equal(a, b) for a, b in zip(out[0], out[1]))


def _expected_uneven_status(n, n_coeffs, deg, off):
    """The documented rule of rd_roots_uneven for malformed batches: per
    polynomial (consistent offsets whose roots fit the n_coeffs - n root
    array; degree 1..12), then the total of the solvable ones against n_coeffs.
    Returns (status or -1 for "solved", NaN-root mask, overflow)."""
    cons = np.array([(off[i] >= i) and (off[i + 1] >= off[i]) and (off[i + 1] <= n_coeffs - (n - 1 - i))
                     and (off[i + 1] - off[i] == int(deg[i]) + 1) for i in range(n)])
    solvable = cons & (deg >= 1) & (deg <= 12)
    overflow = int(((deg.astype(np.int64) + 1) * solvable).sum()) > n_coeffs
    status = np.where(solvable & (not overflow), -1, 3)
    nan_roots = cons & (~solvable | overflow)
    return status, nan_roots, overflow


@pytest.mark.parametrize("case", ["overlapping", "repeated", "below_index", "tail_too_long", "random"])
def test_malformed_offsets_stay_in_bounds(dev, case):
    """Offsets that are not monotone, or whose ranges overlap, never make the
    uneven path write outside its workspace or the root array: the workspace
    and the root array each sit inside a larger buffer filled with a guard
    pattern, which must come back untouched, and the statuses follow the
    documented rule."""
    rng = np.random.default_rng(["overlapping", "repeated", "below_index", "tail_too_long", "random"].index(case))
    if case == "overlapping":   # polynomials 0, 2, 3 consistent alone, 21 coefficients > 20
        deg, off, n_coeffs = np.array([6, 6, 6, 6]), np.array([0, 7, 3, 10, 17]), 20
    elif case == "repeated":    # the same range again and again
        deg, off, n_coeffs = np.array([6, 6, 6, 6]), np.array([0, 7, 0, 7, 0]), 28
    elif case == "below_index":  # polynomial 2 starts at 1 < 2: its root 0 would be at -1
        deg, off, n_coeffs = np.array([0, 0, 6, 3]), np.array([0, 1, 1, 8, 12]), 12
    elif case == "tail_too_long":  # polynomial 0 fills the array, polynomial 1 has nothing
        deg, off, n_coeffs = np.array([6, 0]), np.array([0, 7, 7]), 7
    else:
        n = 64
        deg = rng.choice([1, 2, 3, 6, 12], size=n)
        off = np.zeros(n + 1, np.int64)
        off[1:] = np.cumsum(deg + 1)
        n_coeffs = int(off[-1])
        for _ in range(6):  # move a few ranges onto others
            i = int(rng.integers(1, n))
            off[i] = int(rng.integers(0, n_coeffs))
    deg = deg.astype(np.uint8)
    off = off.astype(np.int64)
    n = deg.size
    want, nan_mask, overflow = _expected_uneven_status(n, n_coeffs, deg, off)
    assert overflow == (case in ("overlapping",)) or case == "random"
    coeffs = (rng.standard_normal(n_coeffs) + 1j * rng.standard_normal(n_coeffs)).astype(np.complex64)
    need = api.uneven_workspace_bytes(n, n_coeffs)
    guard = 1 << 16
    ws_buf = torch.full((need + guard,), 0xA5, dtype=torch.uint8, device=dev)
    n_roots = n_coeffs - n
    sentinel = complex(7.0, -7.0)
    roots_buf = torch.full((max(n_roots, 0) + 4096,), sentinel, dtype=torch.complex128, device=dev)
    status = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    stats = api.new_stats(dev)
    hist = api.new_hist(W, H, dev)
    L = api.N.load()
    import ctypes
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    c_t, d_t, o_t = (torch.from_numpy(x).to(dev) for x in (coeffs, deg, off))
    prm = api.params("mixed")
    win = WIN3.c()
    rc = L.rd_roots_uneven(p(c_t), api.N.C64, p(d_t), p(o_t), n, n_coeffs, api.N.MIXED, ctypes.byref(prm), None,
                           ctypes.byref(win), W, H, p(hist), p(roots_buf), p(status), p(stats), p(ws_buf), need,
                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.rd_last_error()
    torch.cuda.synchronize()
    assert torch.all(ws_buf[need:] == 0xA5), "write past the workspace"
    r = roots_buf.cpu().numpy()
    assert np.all(r[max(n_roots, 0):] == sentinel), "write past the root array"
    s = status.cpu().numpy()
    assert np.all(s[want == 3] == 3), (s, want)
    assert np.all(s[want == -1] <= 2), (s, want)
    solved_slots = set()
    for i in np.nonzero(want == -1)[0]:
        solved_slots.update(range(off[i] - i, off[i] - i + int(deg[i])))
    for i in range(n):
        slots = list(range(off[i] - i, off[i] - i + int(deg[i])))
        if nan_mask[i] and not solved_slots.intersection(slots):
            assert np.all(np.isnan(r[slots])), i  # nothing solved writes there
        if want[i] == -1:
            assert np.all(np.isfinite(r[slots])), i
    st = api.stats_dict(stats)
    assert st["polys"] == n and st["status_degenerate"] == int((s == 3).sum())


@pytest.mark.parametrize("polish", ["fp64", "df"])
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_warp_specialised_bins_bit_identical_to_one_role_bins(dev, polish, dtype):
    """Degree bins 2..8 in warp-specialised CTAs (rd_uneven_tuning.polish_warps)
    give the one-role bins' roots, status, image and counters bit for bit;
    degrees 9..12 stay one-role in both runs."""
    n = 30000 + 11
    packed, deg, off = WL.uneven_gaussian(5, n, dtype=np.complex64 if dtype == torch.complex64 else np.complex128)
    c_t, d_t, o_t = (torch.from_numpy(x).to(dev) for x in (packed, deg, off))
    ws = api.new_uneven_workspace(n, packed.size, dtype, dev)
    p = api.params("mixed", polish_mode=polish)
    shapes = {d: ((512, 8) if d <= 6 else (256, 4)) for d in range(2, 9)}
    tunings = {"one_role": api.uneven_tuning(block={d: 128 for d in range(2, 13)}),
               "ws": api.uneven_tuning(block={d: (shapes[d][0] if d in shapes else 128) for d in range(2, 13)},
                                       polish_warps={d: v[1] for d, v in shapes.items()})}
    out = {}
    for name, t in tunings.items():
        hist = api.new_hist(W, H, dev)
        stats = api.new_stats(dev)
        roots, status = api.roots_uneven(c_t, d_t, o_t, ws, mode="mixed", params_=p, tuning=t, window=WIN3,
                                         hist=hist, stats=stats)
        torch.cuda.synchronize()
        out[name] = (torch.view_as_real(roots).view(torch.int64).cpu(), status.cpu(), hist.cpu(),
                     api.stats_dict(stats))
    a, b = out["one_role"], out["ws"]
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    assert a[3] == b[3] and b[3]["wait_timeouts"] == 0 and b[3]["polys"] == n


def test_warp_specialised_bins_argument_checks(dev):
    packed, deg, off = WL.uneven_gaussian(3, 100)
    ws = api.new_uneven_workspace(100, packed.size, torch.complex64, dev)
    args = [torch.from_numpy(x).to(dev) for x in (packed, deg, off)]
    for kw, mode in ((dict(polish_warps={9: 2}, block={9: 256}), "mixed"),    # degree above 8
                     (dict(polish_warps={6: 2}, block={6: 128}), "plain"),    # needs RD_MIXED
                     (dict(polish_warps={6: 4}, block={6: 128}), "mixed"),    # no sweep warp left
                     (dict(polish_warps={7: 2}, block={7: 512}), "mixed")):   # degree 7: at most 256 threads
        with pytest.raises(api.N.RootDensityError):
            api.roots_uneven(*args, ws, mode=mode, tuning=api.uneven_tuning(**kw))
