"""The seeded generators: SplitMix64 reference values, counter addressing and
the torch version's bit-equality with the numpy one."""
import numpy as np
import torch

from paper_2507_02164_gb300 import workloads as W


def test_splitmix64_published_sequence():
    """SplitMix64 from state 0 (Steele et al.; Vigna's reference splitmix64.c):
    the first outputs are 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f."""
    z = np.array([1, 2, 3], dtype=np.uint64) * W.GAMMA
    out = W._mix(z)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_addressing_reproduces_subsamples():
    full = W.littlewood(2, 5000)
    idx = np.array([0, 17, 4095, 4999], dtype=np.uint64)
    assert np.array_equal(W.littlewood(2, idx), full[idx.astype(int)])
    c, r = W.unit_disk_roots(1, 300)
    c2, r2 = W.unit_disk_roots(1, np.array([299], dtype=np.uint64))
    assert np.array_equal(c[299:], c2) and np.array_equal(r[299:], r2)


def test_littlewood_values_and_soa_layout():
    a = W.littlewood(2, 10000)
    assert set(np.unique(a)) <= {1, -1, 1j, -1j}
    s = W.littlewood_soa(2, 10000)
    assert np.array_equal(s, a.T)
    # the four values are equally likely
    counts = np.array([(a == v).sum() for v in (1, -1, 1j, -1j)])
    assert counts.min() > 0.23 * a.size


def test_torch_generator_matches_numpy():
    t = W.littlewood_soa_torch(2, 123, 4000, "cpu").numpy()
    ref = W.littlewood(2, np.arange(123, 4123, dtype=np.uint64)).T
    assert np.array_equal(t, ref)


def test_unit_disk_roots_expand_to_coefficients():
    c, r = W.unit_disk_roots(3, 200)
    assert np.all(np.abs(r) < 1)
    for i in range(200):
        assert np.allclose(np.poly(r[i])[::-1], c[i], atol=1e-13)


def test_uneven_batch_layout():
    packed, deg, off = W.uneven_gaussian(3, 1000)
    assert deg.min() == 2 and deg.max() == 12
    assert off[-1] == packed.size and np.all(np.diff(off) == deg.astype(np.int64) + 1)
    # polynomial 5 regenerated alone has the same coefficients
    p5, d5, o5 = W.uneven_gaussian(3, np.array([5], dtype=np.uint64))
    assert np.array_equal(p5, packed[off[5]:off[6]])


def test_tiles_grid():
    c, rho, w, h = W.tiles()
    assert c.size == 480 * 270 and abs(w - 1 / 60) < 1e-15 and abs(h - 1 / 60) < 1e-15
    assert abs(rho - 0.5 * np.hypot(1 / 60, 1 / 60)) < 1e-15
    assert abs(c[0] - (-4 + 0.5 / 60 + 1j * (2.25 - 0.5 / 60))) < 1e-12


def test_torch_uneven_batch_matches_numpy():
    import torch
    packed_t, deg_t, off_t = W.uneven_gaussian_torch(3, 100, 2000, "cpu", dtype=torch.complex128)
    packed, deg, off = W.uneven_gaussian(3, np.arange(100, 2100, dtype=np.uint64), dtype=np.complex128)
    assert np.array_equal(deg_t.numpy(), deg) and np.array_equal(off_t.numpy(), off)
    assert np.allclose(packed_t.numpy(), packed, rtol=1e-14, atol=1e-14)
