"""The soft-density image (CPU): normalisation, continuity at the 3-sigma
cut, chunking, and agreement with a direct per-pixel sum."""
import math

import numpy as np
import torch

from paper_2507_02164_gb300 import splat as SP


def test_single_root_bump_matches_direct_sum():
    z = torch.tensor([0.123 - 0.456j], dtype=torch.complex128)
    img = SP.splat(z).numpy()
    xmin, xmax, ymin, ymax = SP.WINDOW
    px = (xmax - xmin) / SP.W_IMG
    py = (ymax - ymin) / SP.H_IMG
    ix, iy = np.meshgrid(np.arange(SP.W_IMG), np.arange(SP.H_IMG))
    cx = xmin + (ix + 0.5) * px
    cy = ymax - (iy + 0.5) * py
    r2 = ((0.123 - cx) / px) ** 2 + ((-0.456 - cy) / py) ** 2
    ref = np.maximum(0.0, np.exp(-r2 / (2 * SP.SIGMA ** 2)) - math.exp(-4.5))
    assert np.allclose(img, ref, atol=1e-15)


def test_chunking_and_normalisation():
    g = np.random.default_rng(0)
    z = torch.from_numpy(g.uniform(-2, 2, 5000) + 1j * g.uniform(-1.1, 1.1, 5000))
    a = SP.splat(z, chunk=1 << 20)
    b = SP.splat(z, chunk=777)
    assert torch.allclose(a, b, atol=1e-15)
    assert abs(float(SP.splat(z, n_norm=1).sum()) / float(a.sum()) - 5000) < 1e-6


def test_loss_is_continuous_in_the_roots():
    z = torch.tensor([0.3 + 0.1j, -1.2 + 0.7j], dtype=torch.complex128)
    T = torch.zeros(SP.H_IMG, SP.W_IMG, dtype=torch.float64)
    l0 = float(SP.loss(z, T))
    for eps in (1e-9, 1e-7):
        assert abs(float(SP.loss(z + eps, T)) - l0) < 1e3 * eps
