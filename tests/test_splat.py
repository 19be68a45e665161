"""The soft-density image (CPU side): the Python entry refuses CPU tensors
(the image is made by the CUDA kernels only), and the C entry points check
their arguments before touching the device."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2507_02164_gb300 import _native as N
from paper_2507_02164_gb300 import splat as SP


def test_splat_needs_cuda_complex128_roots():
    with pytest.raises(ValueError):
        SP.splat(torch.zeros(4, dtype=torch.complex128))
    with pytest.raises(ValueError):
        SP.splat(np.zeros(4, complex))


def test_splat_argument_validation_without_gpu():
    L = N.load()
    null = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(256)
    w = N.Window(*SP.WINDOW)

    def err(rc):
        return rc, L.rd_last_error().decode()

    for sigma in (0.0, -1.0, 2.5, float("nan")):
        rc, msg = err(L.rd_splat(fake, 4, w, 256, 144, sigma, 1.0, 0, fake, null))
        assert rc == N.RD_EINVAL and "sigma" in msg
    rc, msg = err(L.rd_splat(fake, 4, N.Window(1.0, -1.0, 0.0, 1.0), 256, 144, 1.5, 1.0, 0, fake, null))
    assert rc == N.RD_EINVAL and "window" in msg
    rc, msg = err(L.rd_splat(fake, 4, w, 0, 144, 1.5, 1.0, 0, fake, null))
    assert rc == N.RD_EINVAL and "size" in msg
    rc, msg = err(L.rd_splat(ctypes.c_void_p(8), 4, w, 256, 144, 1.5, 1.0, 0, fake, null))
    assert rc == N.RD_EINVAL and "roots" in msg
    rc, msg = err(L.rd_splat(fake, 4, w, 256, 144, 1.5, 1.0, 0, null, null))
    assert rc == N.RD_EINVAL and "img" in msg
    rc, msg = err(L.rd_splat(fake, 4, w, 256, 144, 1.5, -1.0, 0, fake, null))
    assert rc == N.RD_EINVAL and "scale" in msg
    rc, msg = err(L.rd_splat(fake, -1, w, 256, 144, 1.5, 1.0, 0, fake, null))
    assert rc == N.RD_EINVAL
    assert L.rd_splat(null, 0, w, 256, 144, 1.5, 1.0, 0, fake, null) == 0  # nothing to do
    rc, msg = err(L.rd_splat_backward(fake, 4, w, 256, 144, 1.5, 1.0, 0, null, fake, null))
    assert rc == N.RD_EINVAL and "grad_img" in msg
    rc, msg = err(L.rd_splat_backward(fake, 4, w, 256, 144, 1.5, 1.0, 0, fake, ctypes.c_void_p(8), null))
    assert rc == N.RD_EINVAL and "grad_roots" in msg
    rc, msg = err(L.rd_splat(fake, 4, w, 256, 144, 1.5, 1.0, 2, fake, null))
    assert rc == N.RD_EINVAL and "precision" in msg
