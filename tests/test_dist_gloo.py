"""The sharded multi-rank path on CPU: two gloo ranks each bin their own
shard of the Littlewood stream (with the oracle standing in for the GPU
kernel), the images are summed once, and the result equals the single-process
image of the whole range. A rank that fails before the exchange is detected
by its peer through a short process-group timeout, not a hang."""
from __future__ import annotations

import datetime
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

N_PER_RANK = 3000
WIN = (-2.0, 2.0, -1.125, 1.125)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _image_for(start, stop):
    import oracle
    from paper_2507_02164_gb300 import workloads as WL
    co = WL.littlewood(2, np.arange(start, stop, dtype=np.uint64)).astype(np.complex128)
    roots, _, _, _ = oracle.solve(co, threads=1)
    h, oow = oracle.hist(roots, WIN, 192, 108)
    return h, oow


def _worker(rank, world, port, out_dir, fail_rank):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    from paper_2507_02164_gb300 import dist as D
    try:
        start, stop = D.shard_range(N_PER_RANK, rank)
        h, oow = _image_for(start, stop)
        if rank == fail_rank:
            raise RuntimeError("injected failure before the exchange")
        img = torch.from_numpy(h.view(np.int32).copy())
        D.reduce_images(img, dst=0)
        t = D.max_over_ranks(float(rank + 1))
        if rank == 0:
            np.save(os.path.join(out_dir, "image.npy"), img.numpy().view(np.uint32))
            np.save(os.path.join(out_dir, "tmax.npy"), np.array([t]))
    except RuntimeError as e:
        with open(os.path.join(out_dir, f"error{rank}.txt"), "w") as f:
            f.write(str(e))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, fail_rank, tmp_path):
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, str(tmp_path), fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert not p.is_alive(), "a rank hung"


def test_two_ranks_sum_their_shards(tmp_path):
    _run(2, -1, tmp_path)
    img = np.load(tmp_path / "image.npy")
    ref, _ = _image_for(0, 2 * N_PER_RANK)
    assert np.array_equal(img, ref)
    assert np.load(tmp_path / "tmax.npy")[0] == 2.0


def test_rank_failure_is_reported_not_hung(tmp_path):
    _run(2, 1, tmp_path)
    assert (tmp_path / "error1.txt").exists()
    # rank 0 waited in the reduce and got an error from the process group
    assert (tmp_path / "error0.txt").exists() or not (tmp_path / "image.npy").exists()


def test_shard_ranges_are_disjoint_and_cover():
    from paper_2507_02164_gb300 import dist as D
    rs = [D.shard_range(10, r) for r in range(4)]
    assert rs == [(0, 10), (10, 20), (20, 30), (30, 40)]
    with pytest.raises(ValueError):
        D.shard_range(-1, 0)


# ----------------------------------- differentiation workload across ranks

def _density_worker(rank, world, port, out_dir):
    """Each rank: a leaf x_r, its image D_r = M_r x_r (a differentiable stand-in
    for the soft-density splat, which runs on the GPU), the global image
    sum_r D_r through dist.global_density, the loss |x_r|^2 + sum (D - T)^2,
    and the backward pass."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    from paper_2507_02164_gb300 import dist as D
    try:
        g = torch.Generator().manual_seed(100 + rank)
        M = torch.randn(20, 3, generator=g, dtype=torch.float64)
        x = torch.randn(3, generator=g, dtype=torch.float64).requires_grad_(True)
        img = D.global_density((M @ x).reshape(4, 5))
        T = torch.linspace(0.0, 1.0, 20, dtype=torch.float64).reshape(4, 5)
        L = (x ** 2).sum() + ((img - T) ** 2).sum()
        L.backward()
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), M=M.numpy(), x=x.detach().numpy(),
                 grad=x.grad.numpy(), img=img.detach().numpy())
    finally:
        dist.destroy_process_group()


def test_global_density_gradients_across_two_ranks(tmp_path):
    """The summed image is the same on both ranks, and each rank's gradient
    equals that of the global loss sum_r |x_r|^2 + sum (sum_r M_r x_r - T)^2
    computed in one process."""
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_density_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert not p.is_alive() and p.exitcode == 0
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    D = sum(r["M"] @ r["x"] for r in res)
    T = np.linspace(0.0, 1.0, 20)
    for r in res:
        assert np.allclose(r["img"].reshape(-1), D, rtol=0, atol=1e-14)
        ref = 2 * r["x"] + 2 * r["M"].T @ (D - T)
        assert np.allclose(r["grad"], ref, rtol=1e-13, atol=1e-13)


def test_global_density_is_the_identity_in_one_process():
    from paper_2507_02164_gb300 import dist as D
    x = torch.ones(3, requires_grad=True)
    assert D.global_density(x) is x
