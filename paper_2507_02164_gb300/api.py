"""Python binding of libroots over torch tensors.

PyTorch supplies device memory and the current CUDA stream; every step of the
computation runs in the library's CUDA kernels. Layouts follow
include/rootdensity.h: uniform-degree batches are coefficient-major,
``coeffs[k, i]`` is a_k of polynomial i (shape [d+1, n]) and ``roots[j, i]``
is root j of polynomial i (shape [d, n], complex128).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _native as N


@dataclass(frozen=True)
class Window:
    xmin: float
    xmax: float
    ymin: float
    ymax: float

    def c(self) -> N.Window:
        return N.Window(self.xmin, self.xmax, self.ymin, self.ymax)

    def tuple(self):
        return (self.xmin, self.xmax, self.ymin, self.ymax)


MODES = {"plain": N.PLAIN_FP64, "plain_fp64": N.PLAIN_FP64, "mixed": N.MIXED}
DTYPES = {torch.complex64: N.C64, torch.complex128: N.C128}


def _mode(mode) -> int:
    return MODES[mode] if isinstance(mode, str) else int(mode)


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check_cuda(name: str, t: torch.Tensor, dtype=None, contiguous=True):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if contiguous and not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def params(mode="mixed", **overrides) -> N.Params:
    """rd_params with the library defaults for `mode`, then `overrides` applied."""
    p = N.default_params(_mode(mode))
    for k, v in overrides.items():
        if k == "shift" and isinstance(v, str):
            v = {"wilkinson": N.SHIFT_WILKINSON, "rayleigh": N.SHIFT_RAYLEIGH}[v]
        if k == "polish_mode" and isinstance(v, str):
            v = {"fp64": N.POLISH_FP64, "df": N.POLISH_DF}[v]
        setattr(p, k, v)
    return p


def new_stats(device="cuda") -> torch.Tensor:
    """A zeroed rd_stats block (int64 words, read as unsigned)."""
    return torch.zeros(N.STATS_WORDS, dtype=torch.int64, device=device)


def stats_dict(stats: torch.Tensor) -> dict:
    vals = stats.cpu().tolist()
    return dict(zip(N.STATS_FIELDS, vals))


def _check_input(name: str, t: torch.Tensor, dtype=None):
    """An input array the kernels read: a CUDA tensor, or a page-locked CPU
    tensor mapped into the device address space (the kernels then read it
    across the host link, zero copy), checked through the CUDA runtime."""
    if not t.is_cuda:
        if not (t.is_pinned() and N.load().rd_pointer_is_device_accessible(ctypes.c_void_p(t.data_ptr())) == 1):
            raise ValueError(f"{name} must be a CUDA tensor or page-locked host memory mapped for the device")
    _check_cuda(name, t, dtype) if t.is_cuda else None
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _out_device(t: torch.Tensor) -> torch.device:
    """Where outputs go for input t: its GPU, or the current GPU for host input."""
    return t.device if t.is_cuda else torch.device("cuda", torch.cuda.current_device())


def _coeff_args(coeffs: torch.Tensor):
    _check_input("coeffs", coeffs)
    if coeffs.dtype not in DTYPES:
        raise ValueError("coeffs must be complex64 or complex128")
    if coeffs.dim() != 2 or coeffs.shape[0] < 2:
        raise ValueError("coeffs must have shape [degree+1, n]")
    return DTYPES[coeffs.dtype], coeffs.shape[0] - 1, coeffs.shape[1]


def roots_batched(coeffs: torch.Tensor, mode="mixed", params_=None, roots=None, status=None, stats=None,
                  want_roots=True, want_status=True, stream=None):
    """Roots of every column of coeffs ([d+1, n]; on the GPU or in page-locked
    host memory). Returns (roots [d, n] c128, status [n] u8) on the GPU."""
    dt, d, n = _coeff_args(coeffs)
    dev = _out_device(coeffs)
    if want_roots and roots is None:
        roots = torch.empty((d, n), dtype=torch.complex128, device=dev)
    if want_status and status is None:
        status = torch.empty(n, dtype=torch.uint8, device=dev)
    p = params_ if params_ is not None else params(mode)
    N.call("rd_roots_batched", _ptr(coeffs), dt, d, n, _mode(mode), ctypes.byref(p), _ptr(roots),
           _ptr(status), _ptr(stats), _stream(stream))
    return roots, status


def hist_clear(t: torch.Tensor, stream=None):
    _check_cuda("buffer", t)
    words = t.numel() * t.element_size() // 4
    N.call("rd_hist_clear", _ptr(t), words, _stream(stream))
    return t


def new_hist(W=1920, H=1080, device="cuda") -> torch.Tensor:
    h = torch.empty((H, W), dtype=torch.int32, device=device)
    return hist_clear(h)


def make_clip(centres: torch.Tensor, radius: float, nx: int, ny: int, tiles: Window, tile_index=None):
    _check_cuda("centres", centres, torch.complex128)
    c = N.Clip()
    c.centres = centres.data_ptr()
    c.radius = float(radius)
    c.tile_index = tile_index.data_ptr() if tile_index is not None else None
    c.nx, c.ny = nx, ny
    c.tiles = tiles.c()
    return c


def roots_density(coeffs: torch.Tensor, window: Window, hist: torch.Tensor, mode="mixed", params_=None,
                  clip=None, roots=None, status=None, stats=None, stream=None):
    """Fused roots + binning into hist ([H, W] int32 viewed as uint32, accumulated).
    coeffs may be on the GPU or in page-locked host memory (read by the kernel
    across the host link)."""
    dt, d, n = _coeff_args(coeffs)
    _check_cuda("hist", hist)
    H, W = hist.shape
    p = params_ if params_ is not None else params(mode)
    N.call("rd_roots_density", _ptr(coeffs), dt, d, n, _mode(mode), ctypes.byref(p),
           ctypes.byref(clip) if clip is not None else None, window.c(), W, H, _ptr(hist), _ptr(roots),
           _ptr(status), _ptr(stats), _stream(stream))
    return hist


def density_accumulate(roots: torch.Tensor, window: Window, hist: torch.Tensor, status=None, clip=None,
                       stats=None, stream=None):
    """Bin roots (complex128) into hist ([H, W] int32 viewed as uint32, accumulated).
    roots [d, n] is a solve's output for n polynomials; a 1-D tensor stands
    alone. status ([n] uint8) keeps only the roots of polynomials with status
    OK; clip (make_clip) maps each root w of polynomial i to c_i + rho w and
    keeps it only inside polynomial i's own tile."""
    _check_cuda("roots", roots, torch.complex128)
    _check_cuda("hist", hist)
    if roots.dim() == 2:
        n_polys = roots.shape[1]
    elif roots.dim() == 1:
        n_polys = 0
    else:
        raise ValueError("roots must be [d, n] or 1-D")
    if status is not None:
        _check_cuda("status", status, torch.uint8)
        if n_polys == 0 or status.numel() != n_polys:
            raise ValueError("status needs roots of shape [d, n] and n entries")
    if clip is not None and n_polys == 0:
        raise ValueError("clip needs roots of shape [d, n]")
    H, W = hist.shape
    N.call("rd_density_accumulate", _ptr(roots), _ptr(status), roots.numel(), n_polys, window.c(), W, H,
           ctypes.byref(clip) if clip is not None else None, _ptr(hist), _ptr(stats), _stream(stream))
    return hist


def uneven_workspace_bytes(n: int, n_coeffs: int, dtype=torch.complex64) -> int:
    return int(N.load().rd_uneven_workspace_bytes(n, n_coeffs, DTYPES[dtype]))


def new_uneven_workspace(n: int, n_coeffs: int, dtype=torch.complex64, device="cuda") -> torch.Tensor:
    """A device scratch buffer for roots_uneven (torch allocations are 256-byte aligned)."""
    return torch.empty(uneven_workspace_bytes(n, n_coeffs, dtype), dtype=torch.uint8, device=device)


def uneven_tuning(block=None, ctas_per_sm=None, lanes=None, polish_warps=None) -> N.UnevenTuning:
    """rd_uneven_tuning from {degree: value} dicts (missing degrees: defaults;
    polish_warps > 0 runs that degree's bin warp-specialised, degrees <= 8)."""
    t = N.UnevenTuning()
    for arr, vals in ((t.block, block), (t.ctas_per_sm, ctas_per_sm), (t.lanes, lanes),
                      (t.polish_warps, polish_warps)):
        for d, v in (vals or {}).items():
            if not 1 <= int(d) <= 12:
                raise ValueError(f"tuning degree {d} outside 1..12")
            arr[int(d)] = int(v)
    return t


def roots_uneven(coeffs: torch.Tensor, degrees: torch.Tensor, offsets: torch.Tensor, workspace: torch.Tensor,
                 mode="mixed", params_=None, tuning=None, window: Window | None = None, hist=None, roots=None,
                 status=None, stats=None, stream=None, want_roots=True, want_status=True):
    """Roots of a packed uneven-degree batch (coefficients lowest power first,
    polynomial i at coeffs[offsets[i]:offsets[i+1]]); roots packed without the
    leading coefficient. Optionally bins them into hist over window. The
    inputs (coeffs, degrees, offsets) may be on the GPU or in page-locked host
    memory; workspace and outputs are on the GPU."""
    _check_input("coeffs", coeffs)
    if coeffs.dtype not in DTYPES or coeffs.dim() != 1:
        raise ValueError("coeffs must be a 1-D complex64/complex128 tensor")
    _check_input("degrees", degrees, torch.uint8)
    _check_input("offsets", offsets, torch.int64)
    _check_cuda("workspace", workspace)
    n = degrees.numel()
    if offsets.numel() != n + 1:
        raise ValueError("offsets must have n+1 entries")
    ncoef = coeffs.numel()
    dev = workspace.device
    if roots is None and want_roots:
        roots = torch.empty(ncoef - n, dtype=torch.complex128, device=dev)
    if status is None and want_status:
        status = torch.empty(n, dtype=torch.uint8, device=dev)
    p = params_ if params_ is not None else params(mode)
    H, W = hist.shape if hist is not None else (0, 0)
    win = ctypes.byref(window.c()) if window is not None else None
    N.call("rd_roots_uneven", _ptr(coeffs), DTYPES[coeffs.dtype], _ptr(degrees), _ptr(offsets), n, ncoef,
           _mode(mode), ctypes.byref(p), ctypes.byref(tuning) if tuning is not None else None, win, W, H,
           _ptr(hist), _ptr(roots), _ptr(status), _ptr(stats), _ptr(workspace),
           workspace.numel() * workspace.element_size(), _stream(stream))
    return roots, status


def roots_backward(coeffs: torch.Tensor, roots: torch.Tensor, grad_roots: torch.Tensor, status=None,
                   stream=None):
    """grad_coeffs [d+1, n] (dtype of coeffs) from grad_roots [d, n] (complex128)."""
    dt, d, n = _coeff_args(coeffs)
    _check_cuda("roots", roots, torch.complex128)
    _check_cuda("grad_roots", grad_roots, torch.complex128)
    grad = torch.empty_like(coeffs)
    N.call("rd_roots_backward", _ptr(coeffs), dt, d, n, _ptr(roots), _ptr(grad_roots), _ptr(grad),
           _ptr(status), _stream(stream))
    return grad


def roots_backward_uneven(coeffs: torch.Tensor, degrees: torch.Tensor, offsets: torch.Tensor, roots: torch.Tensor,
                          grad_roots: torch.Tensor, grad_coeffs=None, status=None, stream=None):
    """Adjoint of a packed uneven-degree batch (the layout of roots_uneven):
    grad_coeffs (packed like coeffs, same dtype) from grad_roots (packed like
    roots, complex128)."""
    _check_cuda("coeffs", coeffs)
    if coeffs.dtype not in DTYPES or coeffs.dim() != 1:
        raise ValueError("coeffs must be a 1-D complex64/complex128 tensor")
    _check_cuda("degrees", degrees, torch.uint8)
    _check_cuda("offsets", offsets, torch.int64)
    n = degrees.numel()
    if offsets.numel() != n + 1:
        raise ValueError("offsets must have n+1 entries")
    for name, t in (("roots", roots), ("grad_roots", grad_roots)):
        _check_cuda(name, t, torch.complex128)
        if t.numel() != coeffs.numel() - n:
            raise ValueError(f"{name} must have n_coeffs - n entries")
    if grad_coeffs is None:
        grad_coeffs = torch.empty_like(coeffs)
    _check_cuda("grad_coeffs", grad_coeffs, coeffs.dtype)
    N.call("rd_roots_backward_uneven", _ptr(coeffs), DTYPES[coeffs.dtype], _ptr(degrees), _ptr(offsets), n,
           coeffs.numel(), _ptr(roots), _ptr(grad_roots), _ptr(grad_coeffs), _ptr(status), _stream(stream))
    return grad_coeffs


def l2_nodes(nr: int = 16, nt: int = 32):
    """Gauss-Legendre radii and weights on [0, 1] and the angles 2 pi q / nt
    (host lists), from the library: (r, theta, w)."""
    r = (ctypes.c_double * nr)()
    w = (ctypes.c_double * nr)()
    th = (ctypes.c_double * nt)()
    N.call("rd_l2_nodes", nr, nt, ctypes.cast(r, ctypes.c_void_p), ctypes.cast(th, ctypes.c_void_p),
           ctypes.cast(w, ctypes.c_void_p))
    return list(r), list(th), list(w)


def l2_sample_points(nr: int = 16, nt: int = 32, device="cuda") -> torch.Tensor:
    """w_pq = r_p e^{i theta_q} as a [nr*nt] complex128 tensor (index p*nt + q)."""
    r, th, _ = l2_nodes(nr, nt)
    rr = torch.tensor(r, dtype=torch.float64, device=device)
    tt = torch.tensor(th, dtype=torch.float64, device=device)
    return (rr[:, None] * torch.exp(1j * tt)[None, :]).reshape(-1)


def l2_approx(samples: torch.Tensor, nr: int = 16, nt: int = 32, degree: int = 6, coeffs=None, stream=None,
              precision: str = "fp64", centres=None, radius: float = 0.0, clip=None):
    """samples [n, nr*nt] complex128 -> coeffs [degree+1, n] complex128 (local variable w).
    precision "fp64" (FP64 sums) or "df" (double-float sums on the FP32 pipe).
    With clip (an N.Clip whose tile grid the caller sets), centres [n]
    complex128 and radius are checked and written into it: the map z = c + rho w
    that rd_roots_density / density_accumulate apply to the roots."""
    _check_cuda("samples", samples, torch.complex128)
    n = samples.shape[0]
    if samples.shape[1] != nr * nt:
        raise ValueError("samples must have shape [n, nr*nt]")
    if coeffs is None:
        coeffs = torch.empty((degree + 1, n), dtype=torch.complex128, device=samples.device)
    if centres is not None:
        _check_cuda("centres", centres, torch.complex128)
    N.call("rd_l2_approx", _ptr(samples), n, nr, nt, degree, {"fp64": N.L2_FP64, "df": N.L2_DF}[precision],
           _ptr(centres), float(radius), _ptr(coeffs), ctypes.byref(clip) if clip is not None else None,
           _stream(stream))
    return coeffs


def alu_peak(kind: str, iters: int, ctas_per_sm: int = 4, sink=None, stream=None) -> int:
    """Enqueue the library's FMA throughput kernel ("fp32" or "fp64"); returns
    the flops of the launch (the caller times it on `stream`)."""
    if sink is None:
        sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    fl = ctypes.c_uint64(0)
    N.call("rd_alu_peak", {"fp32": N.PEAK_FP32, "fp64": N.PEAK_FP64}[kind], int(iters), int(ctas_per_sm),
           _ptr(sink), ctypes.byref(fl), _stream(stream))
    return int(fl.value)


class RootsFn(torch.autograd.Function):
    """roots = RootsFn.apply(coeffs [d+1, n], mode, params): forward by the QR
    solver (rd_params or None for the defaults), backward by the
    implicit-differentiation adjoint (no QR history kept)."""

    @staticmethod
    def forward(ctx, coeffs, mode="mixed", params_=None):
        roots, status = roots_batched(coeffs.detach().contiguous(), mode=mode, params_=params_)
        ctx.save_for_backward(coeffs, roots)
        ctx.mark_non_differentiable(status)
        return roots, status

    @staticmethod
    def backward(ctx, grad_roots, grad_status):
        coeffs, roots = ctx.saved_tensors
        if grad_roots is None:
            return None, None, None
        g = roots_backward(coeffs.detach().contiguous(), roots, grad_roots.contiguous().to(torch.complex128))
        return g, None, None


def roots(coeffs: torch.Tensor, mode="mixed", params_=None):
    """Differentiable roots: (roots [d, n] complex128, status [n] uint8);
    params_ as in roots_batched (e.g. an autotuned launch shape)."""
    return RootsFn.apply(coeffs, mode, params_)


def field_spec(tiles: Window, nx: int, ny: int, radius: float = 0.0, poly=None, degree: int = 6,
               nr: int = 16) -> N.FieldSpec:
    """rd_field_spec: nx x ny tiles over `tiles`; `poly` (c_0..c_k, k <= 12) for
    f = RD_F_POLY; radius <= 0 means half the tile diagonal."""
    sp = N.FieldSpec()
    sp.tiles = tiles.c()
    sp.nx, sp.ny, sp.radius, sp.nr, sp.degree = nx, ny, float(radius), nr, degree
    if poly is not None:
        c = [complex(v) for v in poly]
        if not 1 <= len(c) <= 13:
            raise ValueError("poly needs 1..13 coefficients")
        sp.poly_degree = len(c) - 1
        for k, v in enumerate(c):
            sp.poly[2 * k], sp.poly[2 * k + 1] = v.real, v.imag
    return sp


def field_density(spec: N.FieldSpec, window: Window, hist: torch.Tensor, f: str = "sin_cube", mode="mixed",
                  params_=None, coeffs=None, roots=None, status=None, stats=None, stream=None):
    """The whole path for f in one launch: f at the 16 x 32 nodes of every
    tile's sub-disk, L2 coefficients, roots, own-tile clip, histogram
    (accumulated into hist [H, W]). Optional outputs: coeffs [7, nx*ny],
    roots [6, nx*ny] (complex128, local variable w), status [nx*ny] uint8."""
    _check_cuda("hist", hist)
    for name, t in (("coeffs", coeffs), ("roots", roots)):
        if t is not None:
            _check_cuda(name, t, torch.complex128)
    H, W = hist.shape
    func = {"sin_cube": N.F_SIN_CUBE, "poly": N.F_POLY}[f]
    p = params_ if params_ is not None else params(mode)
    N.call("rd_field_density", func, ctypes.byref(spec), _mode(mode), ctypes.byref(p), window.c(), W, H,
           _ptr(hist), _ptr(coeffs), _ptr(roots), _ptr(status), _ptr(stats), _stream(stream))
    return hist
