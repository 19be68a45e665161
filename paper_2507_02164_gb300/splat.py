"""Soft root-density loss (Gaussian splat) for differentiating through roots.

A differentiable stand-in for the hard histogram: every root adds a
truncated Gaussian bump to a coarse image, and the image is compared with a
target image. With the roots from ``api.roots`` (the autograd Function whose
backward is the implicit-differentiation adjoint) this gives gradients of a
root-density objective with respect to the polynomial coefficients.

Image: W x H pixel centres over the window (pixel (iy, ix) at
x = xmin + (ix + 0.5) px, y = ymax - (iy + 0.5) py); bump
w(r) = max(0, exp(-r^2 / (2 sigma^2)) - exp(-9/2)), r in pixel units, which
is continuous where it reaches zero at 3 sigma; D = sum_roots w / n_roots.
Loss L = sum_roots |z|^2 + lam * sum_pixels (D - T)^2.
"""
from __future__ import annotations

import math

import torch

WINDOW = (-2.0, 2.0, -1.125, 1.125)
W_IMG, H_IMG = 256, 144
SIGMA = 1.5


def splat(roots: torch.Tensor, window=WINDOW, W: int = W_IMG, H: int = H_IMG, sigma: float = SIGMA,
          n_norm: int | None = None, chunk: int = 1 << 16) -> torch.Tensor:
    """Soft density image [H, W] (float64) of the complex roots (any shape),
    accumulated over chunks of `chunk` roots to bound the stencil buffers."""
    z = roots.reshape(-1)
    norm = float(n_norm if n_norm is not None else z.numel())
    if z.numel() > chunk:
        img = None
        for c0 in range(0, z.numel(), chunk):
            part = _splat_sum(z[c0:c0 + chunk], window, W, H, sigma)
            img = part if img is None else img + part
        return img / norm
    return _splat_sum(z, window, W, H, sigma) / norm


def _splat_sum(z: torch.Tensor, window, W: int, H: int, sigma: float) -> torch.Tensor:
    """Sum of the bumps of the roots z (1-D complex) on the [H, W] grid."""
    xmin, xmax, ymin, ymax = window
    px = (xmax - xmin) / W
    py = (ymax - ymin) / H
    # root position in pixel units, pixel centres at integer + 0.5
    u = (z.real - xmin) / px
    v = (ymax - z.imag) / py
    R = int(math.ceil(3 * sigma)) + 1
    off = torch.arange(-R, R + 1, device=z.device)
    cu = torch.floor(u).detach().long()
    cv = torch.floor(v).detach().long()
    ix = cu[:, None, None] + off[None, None, :]            # [n, 1, 2R+1]
    iy = cv[:, None, None] + off[None, :, None]            # [n, 2R+1, 1]
    du = u[:, None, None] - (ix.to(u.dtype) + 0.5)
    dv = v[:, None, None] - (iy.to(v.dtype) + 0.5)
    w = torch.clamp(torch.exp(-(du * du + dv * dv) / (2 * sigma * sigma)) - math.exp(-4.5), min=0.0)
    inside = (ix >= 0) & (ix < W) & (iy >= 0) & (iy < H) & torch.isfinite(u)[:, None, None] & torch.isfinite(v)[:, None, None]
    w = torch.where(inside, w, torch.zeros_like(w))
    flat = (iy.clamp(0, H - 1) * W + ix.clamp(0, W - 1)).expand_as(w).reshape(-1)
    img = torch.zeros(H * W, dtype=w.dtype, device=z.device).index_add(0, flat, w.reshape(-1))
    return img.reshape(H, W)


def loss(roots: torch.Tensor, target: torch.Tensor, lam: float = 1.0, **kw) -> torch.Tensor:
    """sum |z|^2 + lam * sum (splat(roots) - target)^2."""
    d = splat(roots, **kw)
    return (roots.real ** 2 + roots.imag ** 2).sum() + lam * ((d - target) ** 2).sum()
