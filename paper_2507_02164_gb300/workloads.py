"""Seeded synthetic inputs for the batched root / root-density path.

Every random number is a SplitMix64 output (G. Steele, D. Lea, C. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator, so any polynomial of a batch can be regenerated from
(seed, index) alone without producing the batch:

    key(seed)       = mix(seed + GAMMA)                 (mod 2**64)
    draw(seed, c)   = mix(key(seed) + (c + 1) * GAMMA)  (mod 2**64)
    mix(z)          : z ^= z >> 30; z *= 0xbf58476d1ce4e5b9;
                      z ^= z >> 27; z *= 0x94d049bb133111eb; z ^= z >> 31
    uniform(seed,c) = (draw(seed, c) >> 11) * 2**-53          in [0, 1)

Polynomial i uses counters c = i * STRIDE + j for its j-th draw.

This module holds input recipes only. It does none of the method's
arithmetic: no companion matrix, no QR sweep, no polish, no binning, no
quadrature. Both the CPU oracle and the CUDA library are fed from here.

Recipes (coefficients are stored lowest power first, a_0 .. a_d):

* ``unit_disk_roots``: degree-6 monic polynomials built from 6 roots drawn
  uniformly by area in the unit disk (r = sqrt(U), theta = 2 pi U'), expanded
  in FP64. The roots are returned too, so the true roots are known.
* ``littlewood``: degree-6 polynomials with a_k drawn i.i.d. from
  {1, -1, i, -i} (two bits each of one draw), stored complex64.
* ``gaussian``: degree-d polynomials with Re, Im of every coefficient N(0,1)
  (Box-Muller on two uniforms).
* ``uneven_gaussian``: degree uniform over 2..12, Gaussian coefficients,
  packed poly-major with a u8 degree array and i64 offsets.
* ``tiles``: the tile grid of the full pipeline (centres, radius) for
  f(z) = sin(z^3) + 0.5 z.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = 2.0 ** -53

# draws reserved per polynomial by each recipe
STRIDE_UNIT_DISK = 16
STRIDE_LITTLEWOOD = 1
STRIDE_GAUSSIAN = 32
STRIDE_UNEVEN = 32

LITTLEWOOD_VALUES = np.array([1.0, -1.0, 1.0j, -1.0j], dtype=np.complex128)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    return z ^ (z >> np.uint64(31))


def key(seed: int) -> np.uint64:
    with np.errstate(over="ignore"):
        return _mix(np.array([seed], dtype=np.uint64) + GAMMA)[0]


def draw(seed: int, counters) -> np.ndarray:
    """SplitMix64 output number ``counters`` (0-based) of stream ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key(seed) + (c + np.uint64(1)) * GAMMA)


def uniform(seed: int, counters) -> np.ndarray:
    return (draw(seed, counters) >> np.uint64(11)).astype(np.float64) * _TWO_M53


def _counters(idx: np.ndarray, stride: int, j: int) -> np.ndarray:
    return np.asarray(idx, dtype=np.uint64) * np.uint64(stride) + np.uint64(j)


def _indices(n_or_idx) -> np.ndarray:
    if np.isscalar(n_or_idx):
        return np.arange(int(n_or_idx), dtype=np.uint64)
    return np.asarray(n_or_idx, dtype=np.uint64)


def unit_disk_roots(seed: int, n_or_idx, degree: int = 6):
    """Return (coeffs [n, degree+1] complex128, roots [n, degree] complex128).

    Root k of polynomial i: r = sqrt(U(c=16i+2k)), theta = 2 pi U(c=16i+2k+1).
    The monic polynomial prod_k (z - root_k) is expanded in FP64, multiplying
    the factors in order k = 0, 1, ..., degree-1.
    """
    idx = _indices(n_or_idx)
    n = idx.size
    roots = np.empty((n, degree), dtype=np.complex128)
    for k in range(degree):
        r = np.sqrt(uniform(seed, _counters(idx, STRIDE_UNIT_DISK, 2 * k)))
        th = 2.0 * math.pi * uniform(seed, _counters(idx, STRIDE_UNIT_DISK, 2 * k + 1))
        roots[:, k] = r * np.cos(th) + 1j * (r * np.sin(th))
    c = np.zeros((n, degree + 1), dtype=np.complex128)
    c[:, 0] = 1.0  # running product, highest power last once complete
    # c holds the product of the first k factors, lowest power first, in c[:, :k+1]
    for k in range(degree):
        new = np.zeros_like(c)
        new[:, 1:k + 2] = c[:, 0:k + 1]          # multiply by z
        new[:, 0:k + 1] -= roots[:, k:k + 1] * c[:, 0:k + 1]  # minus root_k times
        c = new
    return c, roots


def littlewood(seed: int, n_or_idx, degree: int = 6, dtype=np.complex64):
    """Coefficients [n, degree+1]: a_k = (1, -1, i, -i)[bits 2k, 2k+1 of draw(seed, i)]."""
    if degree > 31:
        raise ValueError("littlewood: at most 32 two-bit fields per draw")
    idx = _indices(n_or_idx)
    x = draw(seed, _counters(idx, STRIDE_LITTLEWOOD, 0))
    out = np.empty((idx.size, degree + 1), dtype=dtype)
    for k in range(degree + 1):
        sel = ((x >> np.uint64(2 * k)) & np.uint64(3)).astype(np.int64)
        out[:, k] = LITTLEWOOD_VALUES[sel]
    return out


def littlewood_soa(seed: int, n: int, degree: int = 6) -> np.ndarray:
    """Same values as ``littlewood`` but coefficient-major: [degree+1, n] complex64."""
    idx = np.arange(n, dtype=np.uint64)
    x = draw(seed, _counters(idx, STRIDE_LITTLEWOOD, 0))
    out = np.empty((degree + 1, n), dtype=np.complex64)
    table = LITTLEWOOD_VALUES.astype(np.complex64)
    for k in range(degree + 1):
        out[k] = table[((x >> np.uint64(2 * k)) & np.uint64(3)).astype(np.intp)]
    return out


def _normal_pair(seed: int, idx: np.ndarray, stride: int, j: int):
    """Box-Muller: (sqrt(-2 ln(1-U1)) cos 2piU2, sqrt(-2 ln(1-U1)) sin 2piU2)."""
    u1 = uniform(seed, _counters(idx, stride, j))
    u2 = uniform(seed, _counters(idx, stride, j + 1))
    rad = np.sqrt(-2.0 * np.log1p(-u1))
    th = 2.0 * math.pi * u2
    return rad * np.cos(th), rad * np.sin(th)


def gaussian(seed: int, n_or_idx, degree: int = 6, dtype=np.complex128):
    """Coefficients [n, degree+1], Re and Im of a_k from draws 2k, 2k+1."""
    idx = _indices(n_or_idx)
    out = np.empty((idx.size, degree + 1), dtype=np.complex128)
    for k in range(degree + 1):
        re, im = _normal_pair(seed, idx, STRIDE_GAUSSIAN, 2 * k)
        out[:, k] = re + 1j * im
    return out.astype(dtype)


UNEVEN_MIN_DEG = 2
UNEVEN_MAX_DEG = 12


def uneven_degrees(seed: int, n_or_idx) -> np.ndarray:
    """Degree of polynomial i: 2 + floor(11 U(c=32i)), uniform over 2..12."""
    idx = _indices(n_or_idx)
    u = uniform(seed, _counters(idx, STRIDE_UNEVEN, 0))
    return (UNEVEN_MIN_DEG + np.floor(11.0 * u)).astype(np.uint8)


def uneven_gaussian(seed: int, n_or_idx, dtype=np.complex64):
    """Packed uneven-degree batch.

    Returns (coeffs_packed [sum(d_i+1)] dtype, degrees [n] u8, offsets [n+1] i64)
    where polynomial i occupies coeffs_packed[offsets[i]:offsets[i+1]], lowest
    power first; Re, Im of coefficient k use draws 1+2k, 2+2k.
    """
    idx = _indices(n_or_idx)
    deg = uneven_degrees(seed, idx)
    offsets = np.zeros(idx.size + 1, dtype=np.int64)
    np.cumsum(deg.astype(np.int64) + 1, out=offsets[1:])
    packed = np.empty(int(offsets[-1]), dtype=np.complex128)
    for k in range(UNEVEN_MAX_DEG + 1):
        have = deg >= k
        if not np.any(have):
            continue
        re, im = _normal_pair(seed, idx[have], STRIDE_UNEVEN, 1 + 2 * k)
        packed[offsets[:-1][have] + k] = re + 1j * im
    return packed.astype(dtype), deg, offsets


# ---- full-pipeline tiling (no randomness) ---------------------------------

def f_sin_cube(z):
    """f(z) = sin(z^3) + 0.5 z, the full-pipeline target function (numpy or torch)."""
    return np_or_torch_sin(z * z * z) + 0.5 * z


def np_or_torch_sin(z):
    if isinstance(z, np.ndarray) or np.isscalar(z):
        return np.sin(z)
    import torch  # local: only the device sampler path needs it
    return torch.sin(z)


def tiles(xmin=-4.0, xmax=4.0, ymin=-2.25, ymax=2.25, nx=480, ny=270):
    """Tile grid: returns (centres [ny*nx] complex128 row-major from the top-left,
    radius (tile half-diagonal), tile width, tile height). Tile t = iy*nx + ix
    covers [xmin + ix*w, xmin + (ix+1)*w) x (ymax - (iy+1)*h, ymax - iy*h]."""
    w = (xmax - xmin) / nx
    h = (ymax - ymin) / ny
    ix = np.arange(nx, dtype=np.float64)
    iy = np.arange(ny, dtype=np.float64)
    cx = xmin + (ix + 0.5) * w
    cy = ymax - (iy + 0.5) * h
    centres = (cx[None, :] + 1j * cy[:, None]).reshape(-1)
    radius = 0.5 * math.hypot(w, h)
    return centres, radius, w, h


# ---- the same generators as torch ops (any device) -------------------------
# torch has no uint64 arithmetic, so SplitMix64 runs on int64 with wrapping
# multiplication (two's complement) and logical right shifts done by masking;
# the bits equal the numpy version above.

def _to_i64(u: int) -> int:
    return u - (1 << 64) if u >= (1 << 63) else u


def _srl(z, k: int):
    import torch
    return torch.bitwise_and(torch.bitwise_right_shift(z, k), (1 << (64 - k)) - 1)


def _mix_t(z):
    z = torch_xor(z, _srl(z, 30)) * _to_i64(0xBF58476D1CE4E5B9)
    z = torch_xor(z, _srl(z, 27)) * _to_i64(0x94D049BB133111EB)
    return torch_xor(z, _srl(z, 31))


def torch_xor(a, b):
    import torch
    return torch.bitwise_xor(a, b)


def draw_torch(seed: int, counters):
    """draw(seed, counters) for an int64 torch tensor of counters (same bits, as int64)."""
    k = _to_i64(int(key(seed)))
    g = _to_i64(int(GAMMA))
    return _mix_t(k + (counters + 1) * g)


def littlewood_soa_torch(seed: int, start: int, n: int, device, degree: int = 6):
    """Coefficient-major [degree+1, n] complex64 Littlewood batch for indices
    start .. start+n-1, generated on `device` (same values as ``littlewood``)."""
    import torch
    idx = torch.arange(start, start + n, dtype=torch.int64, device=device)
    x = draw_torch(seed, idx * STRIDE_LITTLEWOOD)
    table = torch.tensor([1, -1, 1j, -1j], dtype=torch.complex64, device=device)
    out = torch.empty((degree + 1, n), dtype=torch.complex64, device=device)
    for k in range(degree + 1):
        sel = torch.bitwise_and(_srl(x, 2 * k) if k else x, 3)
        out[k] = table[sel]
    return out


def uniform_torch(seed: int, counters):
    """uniform(seed, counters) as float64 torch values (same values as the numpy version)."""
    import torch
    x = draw_torch(seed, counters)
    return torch.bitwise_and(torch.bitwise_right_shift(x, 11), (1 << 53) - 1).to(torch.float64) * _TWO_M53


def uneven_gaussian_torch(seed: int, start: int, n: int, device, dtype=None):
    """``uneven_gaussian`` for indices start .. start+n-1, generated on `device`.

    Degrees and offsets equal the numpy version exactly; the Gaussian values
    come from the device's log1p / cos / sin and can differ from numpy's in
    the last bits, so parity checks take the stored device values as input.
    Returns (coeffs_packed [sum(d+1)], degrees [n] u8, offsets [n+1] i64).
    """
    import torch
    dtype = dtype or torch.complex64
    idx = torch.arange(start, start + n, dtype=torch.int64, device=device)
    u = uniform_torch(seed, idx * STRIDE_UNEVEN)
    deg = (UNEVEN_MIN_DEG + torch.floor(11.0 * u)).to(torch.int64)
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(deg + 1, dim=0, out=offsets[1:])
    total = int(offsets[-1].item())
    packed = torch.empty(total, dtype=torch.complex128, device=device)
    for k in range(UNEVEN_MAX_DEG + 1):
        have = deg >= k
        sel = idx[have]
        u1 = uniform_torch(seed, sel * STRIDE_UNEVEN + (1 + 2 * k))
        u2 = uniform_torch(seed, sel * STRIDE_UNEVEN + (2 + 2 * k))
        rad = torch.sqrt(-2.0 * torch.log1p(-u1))
        th = 2.0 * math.pi * u2
        packed[offsets[:-1][have] + k] = torch.complex(rad * torch.cos(th), rad * torch.sin(th))
    return packed.to(dtype), deg.to(torch.uint8), offsets
