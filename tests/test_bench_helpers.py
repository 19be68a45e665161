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


def test_within_bar_needs_the_kappa_scaled_bound_and_a_small_excluded_share(orc):
    """within_bar follows the parity tests' bar: the bar on well-conditioned
    roots, 1e-11 max(1, kappa) on every root, and at most 6 % of the roots
    left out as ill-conditioned."""
    co, _ = WL.unit_disk_roots(1, 4000)  # seeded roots in the unit disk: some close pairs
    ref, ref_st, _, _ = orc.solve(co, tol=1e-13)
    ok = np.zeros(co.shape[0], np.uint8)
    s = bench.root_error_summary(ref.copy(), ok, ref, ref_st, co, 1e-9, 1e3)
    assert s["within_bar"] and s["kappa_scaled_ok"] and s["excluded_fraction"] <= 0.06
    # an ill-conditioned root (left out of the bar) moved far beyond 1e-11 kappa fails the bound
    kap = orc.root_condition(co, ref)
    i, j = np.unravel_index(np.argmax(kap), kap.shape)
    assert kap[i, j] > 1e3
    bad = ref.copy()
    bad[i, j] += 1e-11 * kap[i, j] * 100 * max(1.0, abs(ref[i, j]))
    s2 = bench.root_error_summary(bad, ok, ref, ref_st, co, 1e-9, 1e3)
    assert s2["max_rel_err"] <= 1e-9 and not s2["kappa_scaled_ok"] and not s2["within_bar"]
    # a cap that leaves out more than 6 % of the roots fails too
    s3 = bench.root_error_summary(ref.copy(), ok, ref, ref_st, co, 1e-9, 1.0)
    assert s3["excluded_fraction"] > 0.06 and not s3["within_bar"]


def test_launch_plan():
    assert bench.launch_plan(1, {}, "ours") == ("run", 1)
    assert bench.launch_plan(8, {}, "ours") == ("exec", 8)
    assert bench.launch_plan(8, {}, "reference") == ("run", 1)
    assert bench.launch_plan(4, {"WORLD_SIZE": "4"}, "ours") == ("run", 4)
    kind, msg = bench.launch_plan(8, {"WORLD_SIZE": "1"}, "ours")
    assert kind == "error" and "WORLD_SIZE" in msg
    assert bench.launch_plan(0, {}, "ours")[0] == "error"
    argv = bench.torchrun_argv(4, ["--gpus", "4", "--steps", "2"], 29512)
    assert argv[1:4] == ["-m", "torch.distributed.run", "--nnodes=1"]
    assert "--nproc-per-node=4" in argv and "--master-addr=127.0.0.1" in argv and "--master-port=29512" in argv
    assert argv[-4:] == ["--gpus", "4", "--steps", "2"] and argv[-5].endswith("bench.py")


def test_workload_config_labels_the_real_world_size():
    args = bench.parse_args(["--gpus", "4"])
    args.log2n = 26
    assert bench.workload_config(args, 4)["parallelism"] == "dp4"
    assert bench.workload_config(args, 1)["parallelism"] == "dp1"


def test_mismatched_gpus_and_world_size_is_refused():
    import os
    import subprocess
    import sys
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--steps", "1"], cwd=bench.ROOT, env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "WORLD_SIZE" in r.stderr
