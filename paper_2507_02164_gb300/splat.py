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

The image and its pull-back to the roots run in the library's CUDA kernels
(rd_splat, rd_splat_backward), wrapped as an autograd Function.
"""
from __future__ import annotations

import torch

from . import _native as N

WINDOW = (-2.0, 2.0, -1.125, 1.125)
W_IMG, H_IMG = 256, 144
SIGMA = 1.5


def _stream():
    return torch.cuda.current_stream().cuda_stream


PRECISIONS = {"fp64": N.SPLAT_FP64, "fp32": N.SPLAT_FP32}


class SplatFn(torch.autograd.Function):
    """img [H, W] float64 = scale * sum over roots of the truncated bump."""

    @staticmethod
    def forward(ctx, roots, window, W, H, sigma, scale, precision):
        z = roots.detach().reshape(-1).contiguous()
        img = torch.zeros((H, W), dtype=torch.float64, device=z.device)
        win = N.Window(*window)
        N.call("rd_splat", z.data_ptr(), z.numel(), win, W, H, float(sigma), float(scale), precision,
               img.data_ptr(), _stream())
        ctx.save_for_backward(z)
        ctx.args = (win, W, H, float(sigma), float(scale), precision, roots.shape)
        return img

    @staticmethod
    def backward(ctx, grad_img):
        (z,) = ctx.saved_tensors
        win, W, H, sigma, scale, precision, shape = ctx.args
        g = grad_img.detach().to(torch.float64).contiguous()
        out = torch.empty_like(z)
        N.call("rd_splat_backward", z.data_ptr(), z.numel(), win, W, H, sigma, scale, precision, g.data_ptr(),
               out.data_ptr(), _stream())
        return out.reshape(shape), None, None, None, None, None, None


def splat(roots: torch.Tensor, window=WINDOW, W: int = W_IMG, H: int = H_IMG, sigma: float = SIGMA,
          n_norm: int | None = None, precision: str = "fp64") -> torch.Tensor:
    """Soft density image [H, W] (float64) of the complex128 CUDA roots (any
    shape), normalised by n_norm (default: the number of roots). precision
    "fp64" (~1e-14) or "fp32" (the stencil on the FP32 pipe, ~1e-6)."""
    if not (isinstance(roots, torch.Tensor) and roots.is_cuda and roots.dtype == torch.complex128):
        raise ValueError("splat needs a complex128 CUDA tensor of roots")
    norm = float(n_norm if n_norm is not None else roots.numel())
    return SplatFn.apply(roots, tuple(float(v) for v in window), int(W), int(H), float(sigma), 1.0 / norm,
                         PRECISIONS[precision])


def loss(roots: torch.Tensor, target: torch.Tensor, lam: float = 1.0, global_sum=None, **kw) -> torch.Tensor:
    """sum |z|^2 + lam * sum (splat(roots) - target)^2.

    Across ranks: pass n_norm = the number of roots of all ranks and
    global_sum = dist.global_density; the image term then uses the summed
    image and the |z|^2 term is this rank's share (the loss value is the sum
    of the ranks' |z|^2 terms plus one image term; the gradients of every
    rank's roots are those of that global loss)."""
    d = splat(roots, **kw)
    if global_sum is not None:
        d = global_sum(d)
    return (roots.real ** 2 + roots.imag ** 2).sum() + lam * ((d - target) ** 2).sum()
