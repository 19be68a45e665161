"""Host logic of bench.py's root-error report (CPU): per-polynomial root
matching and the error summary against the oracle."""
from __future__ import annotations

import numpy as np

import bench
from paper_2507_02164_gb300 import workloads as WL


def test_match_roots_undoes_any_order_and_resolves_close_pairs():
    rng = np.random.default_rng(1)
    ref = rng.standard_normal((500, 6)) + 1j * rng.standard_normal((500, 6))
    ref[0, 1] = ref[0, 0] + 3e-13  # a nearly double root: nearest pairing is ambiguous there
    perm = np.array([rng.permutation(6) for _ in range(500)])
    gpu = np.take_along_axis(ref, perm, axis=1)
    gpu[0] = ref[0][[1, 0, 2, 3, 4, 5]] + 1e-13
    got = bench.match_roots(gpu, ref)
    assert np.abs(got - ref).max() <= 5e-13


def test_root_error_summary_against_the_oracle(orc):
    idx = np.arange(2000, dtype=np.uint64) * np.uint64(1024)
    co = WL.littlewood(2, idx).astype(np.complex128)
    ref, ref_st, _, _ = orc.solve(co, tol=1e-13)
    rng = np.random.default_rng(2)
    # a stand-in for GPU roots: the oracle's, shuffled, each moved by a relative 1e-12
    noisy = ref * (1 + 1e-12 * np.exp(2j * np.pi * rng.random(ref.shape)))
    gpu = np.take_along_axis(noisy, np.array([rng.permutation(6) for _ in range(idx.size)]), axis=1)
    status = np.zeros(idx.size, np.uint8)
    status[:3] = 2  # REJECTED polynomials are left out of the comparison
    s = bench.root_error_summary(gpu, status, ref, ref_st, co, 1e-9, 1e3)
    assert 5e-13 <= s["max_rel_err"] <= 1.5e-12 * max(1.0, np.abs(ref).max())
    assert s["within_bar"] and s["status_counts"][2] == 3
    assert s["roots_compared"] + s["ill_conditioned_roots"] == 6 * (idx.size - 3)
    # a root off by 1e-6 shows up
    gpu2 = ref.copy()
    gpu2[10, 0] += 1e-6
    s2 = bench.root_error_summary(gpu2, np.zeros(idx.size, np.uint8), ref, ref_st, co, 1e-9, 1e3)
    assert not s2["within_bar"] or s2["ill_conditioned_max_rel_err"] >= 1e-7


def test_newton_move_of_kept_roots():
    """The pipeline's accuracy check: a zero of sin(z^3) + z/2 placed in its
    own tile moves by ~0 under one Newton step on f; a point off the zero
    moves by about its distance; roots outside their tile are not counted."""
    import torch

    from paper_2507_02164_gb300 import workloads as WL
    win = (-4.0, 4.0, -2.25, 2.25)
    centres, rho, _, _ = WL.tiles(*win, 480, 270)
    z = 1.0 + 0.5j
    for _ in range(60):
        z = z - (np.sin(z ** 3) + 0.5 * z) / (3 * z ** 2 * np.cos(z ** 3) + 0.5)
    t = int(np.floor((win[3] - z.imag) * 270 / 4.5)) * 480 + int(np.floor((z.real - win[0]) * 480 / 8.0))
    w = np.full((centres.size, 6), np.nan + 0j)
    w[t, 0] = (z - centres[t]) / rho                     # the zero, in its own tile
    w[t, 1] = (z + 2e-9 - centres[t]) / rho              # 2e-9 off it, same tile
    w[t + 1, 0] = (z - centres[t + 1]) / rho             # the zero, but not in tile t + 1
    out = bench.newton_move_of_kept(torch.from_numpy(np.ascontiguousarray(w.T)), torch.from_numpy(centres), rho,
                                    win, 480, 270)
    assert out["kept_roots"] == 2
    assert 1e-9 <= out["max_newton_move"] <= 4e-9 and out["within_bar"]
