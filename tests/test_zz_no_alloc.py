"""rd_roots_uneven_static: the uneven-degree solve for callers that cannot
allocate device memory (a plugin under a host framework's allocator, a loop
where cudaMalloc would stall the device, a fixed memory budget). It runs on a
scratch array built into the library instead of a caller workspace.

Checked through the C ABI, for complex64 and complex128 storage and both
precision modes: two calls in a row give the same roots (bit for bit),
status, histogram and counters as rd_roots_uneven with a caller workspace
(the second call sees the scratch the first one left behind), and a batch larger
than the built-in scratch is refused with a clear error. This file is
collected last so that a run stopping at its first failure has already run
every other test; it also passes alone in a fresh process.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_2507_02164_gb300 import _native as N
from paper_2507_02164_gb300 import api, workloads as WL
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu

WIN = api.Window(-3.0, 3.0, -1.6875, 1.6875)
W, H = 1920, 1080


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _static_call(coeffs, dtype, degrees, offsets, n, mode, params, window, hist, roots, status, stats):
    L = N.load()
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    win = window.c()
    rc = L.rd_roots_uneven_static(p(coeffs), dtype, p(degrees), p(offsets), n, coeffs.numel(), mode,
                                  ctypes.byref(params), None, ctypes.byref(win), W, H, p(hist), p(roots),
                                  p(status), p(stats), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, L.rd_last_error().decode()


def _bits(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.int64)


@pytest.mark.parametrize("dtype,mode", [(torch.complex64, "mixed"), (torch.complex128, "mixed"),
                                        (torch.complex128, "plain")])
def test_static_scratch_matches_the_workspace_call_on_two_calls_in_a_row(dev, dtype, mode):
    n = 40000
    packed, deg, off = WL.uneven_gaussian(3, n, dtype=np.complex64 if dtype == torch.complex64 else np.complex128)
    c_t = torch.from_numpy(packed).to(dev)
    d_t = torch.from_numpy(deg).to(dev)
    o_t = torch.from_numpy(off).to(dev)
    assert api.uneven_workspace_bytes(n, packed.size, dtype) <= N.STATIC_SCRATCH_BYTES
    params = api.params(mode)
    # the existing entry point, with a workspace the caller allocated
    ws = api.new_uneven_workspace(n, packed.size, dtype, dev)
    ref_hist = api.new_hist(W, H, dev)
    ref_stats = api.new_stats(dev)
    ref_roots, ref_status = api.roots_uneven(c_t, d_t, o_t, ws, mode=mode, params_=params, window=WIN,
                                             hist=ref_hist, stats=ref_stats)
    torch.cuda.synchronize()
    for call in range(2):
        hist = api.new_hist(W, H, dev)
        stats = api.new_stats(dev)
        roots = torch.full_like(ref_roots, complex(np.nan, np.nan))
        status = torch.full_like(ref_status, 255)
        rc, msg = _static_call(c_t, api.DTYPES[dtype], d_t, o_t, n, api._mode(mode), params, WIN, hist, roots,
                               status, stats)
        assert rc == 0, msg
        torch.cuda.synchronize()
        # the same kernels on the same inputs: the same bits
        assert np.array_equal(_bits(roots), _bits(ref_roots)), call
        assert torch.equal(status, ref_status), call
        assert torch.equal(hist, ref_hist), call
        assert api.stats_dict(stats) == api.stats_dict(ref_stats), call


def test_static_scratch_refuses_a_batch_that_does_not_fit(dev):
    n, n_coeffs = 2_000_000, 16_000_000  # about 136 MB of scratch
    assert api.uneven_workspace_bytes(n, n_coeffs) > N.STATIC_SCRATCH_BYTES
    L = N.load()
    null = ctypes.c_void_p(0)
    rc = L.rd_roots_uneven_static(null, N.C64, null, null, n, n_coeffs, N.MIXED, None, None, None, 0, 0,
                                  null, null, null, null, null)
    assert rc == N.RD_EINVAL
    assert "scratch" in L.rd_last_error().decode()
