"""Python access to the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users; the CUDA library and its
Python binding never import this package.

Arrays are numpy, poly-major: coefficients [n, d+1] complex128 (lowest power
first), roots [n, d] complex128.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

OK, NOT_CONVERGED, SINGULAR, DEGENERATE = 0, 1, 2, 3
SHIFT_RAYLEIGH, SHIFT_WILKINSON = 0, 1

# gcc flags: IEEE semantics (no fast-math, no FMA contraction, so x86 and Arm
# give the same bits), OpenMP for the batch loops.
CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas", "-Wno-maybe-uninitialized"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (if stale) and return its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    srcs = [_SRC, os.path.join(_HERE, "oracle.h")]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(s) for s in srcs)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    """Load the oracle. ORACLE_LIB may name another build of oracle.c (the
    mutation test loads deliberately broken copies this way)."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
            P = ctypes.c_void_p
            i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            sig = {
                "or_givens": (None, [P, P, P, P]),
                "or_companion": (None, [P, i32, P]),
                "or_qr_sweep": (None, [P, i32, i32, P]),
                "or_wilkinson_shift": (None, [P, i32, i32, P]),
                "or_solve_one": (i32, [P, i32, f64, i32, i32, i32, P, P]),
                "or_solve_batch": (i32, [P, i64, i32, f64, i32, i32, i32, P, P, P, i32]),
                "or_solve_fixed": (i32, [P, i32, i32, i32, i32, P]),
                "or_hist": (None, [P, i64, f64, f64, f64, f64, i32, i32, P, P]),
                "or_hist_tiled": (None, [P, i64, i32, P, i32, i32, f64, f64, f64, f64, i32, i32, P, P, P]),
                "or_affine": (None, [P, i64, i32, P, f64]),
                "or_gauss_legendre": (i32, [i32, P, P]),
                "or_l2_approx": (i32, [P, i64, i32, i32, i32, P, P, i32]),
                "or_roots_backward": (None, [P, i64, i32, P, P, P, P]),
                "or_root_condition": (None, [P, i64, i32, P, P]),
                "or_splat": (None, [P, i64, f64, f64, f64, f64, i32, i32, f64, f64, P]),
                "or_splat_grad": (None, [P, i64, f64, f64, f64, f64, i32, i32, f64, f64, P, P]),
                "or_max_threads": (i32, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


# ---------------------------------------------------------------- wrappers

def givens(a: complex, b: complex):
    A = _c128([a])
    B = _c128([b])
    c = np.zeros(1, np.complex128)
    s = np.zeros(1, np.complex128)
    lib().or_givens(_p(A), _p(B), _p(c), _p(s))
    return complex(c[0]), complex(s[0])


def companion(b) -> np.ndarray:
    b = _c128(b)
    n = b.size
    A = np.zeros((n, n), np.complex128)
    lib().or_companion(_p(b), n, _p(A))
    return A


def qr_sweep(A: np.ndarray, m: int, shift: complex) -> np.ndarray:
    A = _c128(A).copy()
    s = _c128([shift])
    lib().or_qr_sweep(_p(A), A.shape[0], m, _p(s))
    return A


def wilkinson_shift(A: np.ndarray, m: int) -> complex:
    A = _c128(A)
    s = np.zeros(1, np.complex128)
    lib().or_wilkinson_shift(_p(A), A.shape[0], m, _p(s))
    return complex(s[0])


def solve(coeffs, tol: float = 1e-13, max_its: int = 40, shift: int = SHIFT_RAYLEIGH,
          exc_period: int = 10, threads: int = 0):
    """Roots of every polynomial (rows of coeffs, lowest power first).

    Returns (roots [n, d] complex128, status [n] u8, sweeps [n] i32, threads used).
    """
    coeffs = _c128(coeffs)
    if coeffs.ndim == 1:
        coeffs = coeffs[None, :]
    n, K = coeffs.shape
    d = K - 1
    roots = np.zeros((n, d), np.complex128)
    status = np.zeros(n, np.uint8)
    sweeps = np.zeros(n, np.int32)
    used = lib().or_solve_batch(_p(coeffs), n, d, tol, max_its, shift, exc_period,
                                _p(roots), _p(status), _p(sweeps), threads)
    if used < 0:
        raise ValueError(f"oracle solve: unsupported degree {d}")
    return roots, status, sweeps, used


def solve_fixed(coeffs, T: int = 10, shift: int = SHIFT_RAYLEIGH, exc_period: int = 0):
    """The paper's fixed schedule: T QR steps per eigenvalue, no deflation test.
    Returns (roots [n, d], status [n])."""
    coeffs = _c128(coeffs)
    if coeffs.ndim == 1:
        coeffs = coeffs[None, :]
    n, K = coeffs.shape
    roots = np.zeros((n, K - 1), np.complex128)
    status = np.zeros(n, np.uint8)
    for i in range(n):
        rc = lib().or_solve_fixed(_p(coeffs[i]), K - 1, T, shift, exc_period, _p(roots[i]))
        if rc < 0:
            raise ValueError("oracle solve_fixed: bad degree or T")
        status[i] = rc
    return roots, status


def hist(roots, window, W: int = 1920, H: int = 1080):
    """Root-density histogram [H, W] u32 of all roots, plus the out-of-window count."""
    r = _c128(roots).reshape(-1)
    h = np.zeros((H, W), np.uint32)
    oow = np.zeros(1, np.uint64)
    xmin, xmax, ymin, ymax = window
    lib().or_hist(_p(r), r.size, xmin, xmax, ymin, ymax, W, H, _p(h), _p(oow))
    return h, int(oow[0])


def hist_tiled(roots, tile_of_poly, nx: int, ny: int, window, W: int = 1920, H: int = 1080):
    r = _c128(roots)
    n, d = r.shape
    t = np.ascontiguousarray(tile_of_poly, dtype=np.int64)
    h = np.zeros((H, W), np.uint32)
    oow = np.zeros(1, np.uint64)
    dropped = np.zeros(1, np.uint64)
    xmin, xmax, ymin, ymax = window
    lib().or_hist_tiled(_p(r), n, d, _p(t), nx, ny, xmin, xmax, ymin, ymax, W, H,
                        _p(h), _p(oow), _p(dropped))
    return h, int(oow[0]), int(dropped[0])


def affine(roots, centres, rho: float) -> np.ndarray:
    r = _c128(roots).copy()
    n, d = r.shape
    c = _c128(centres)
    lib().or_affine(_p(r), n, d, _p(c), rho)
    return r


def gauss_legendre(nr: int):
    x = np.zeros(nr)
    w = np.zeros(nr)
    if lib().or_gauss_legendre(nr, _p(x), _p(w)) != 0:
        raise ValueError("gauss_legendre: nr < 1")
    return x, w


def l2_approx(samples, nr: int = 16, nt: int = 32, degree: int = 6, threads: int = 0,
              return_gram: bool = False):
    """Coefficients [n, degree+1] (in the local variable w) from samples [n, nr*nt]."""
    s = _c128(samples)
    if s.ndim == 1:
        s = s[None, :]
    n = s.shape[0]
    assert s.shape[1] == nr * nt
    coeffs = np.zeros((n, degree + 1), np.complex128)
    gram = np.zeros((degree + 1, degree + 1), np.complex128)
    rc = lib().or_l2_approx(_p(s), n, nr, nt, degree, _p(coeffs), _p(gram), threads)
    if rc != 0:
        raise ValueError(f"oracle l2_approx failed ({rc})")
    return (coeffs, gram) if return_gram else coeffs


def l2_nodes(nr: int = 16, nt: int = 32) -> np.ndarray:
    """Sample points w_pq = r_p e^{i 2 pi q / nt}, index p*nt + q."""
    r, _ = gauss_legendre(nr)
    th = 2.0 * np.pi * np.arange(nt) / nt
    return (r[:, None] * np.exp(1j * th)[None, :]).reshape(-1)


def roots_backward(coeffs, roots, grad_roots):
    a = _c128(coeffs)
    z = _c128(roots)
    g = _c128(grad_roots)
    n, K = a.shape
    out = np.zeros((n, K), np.complex128)
    status = np.zeros(n, np.uint8)
    lib().or_roots_backward(_p(a), n, K - 1, _p(z), _p(g), _p(out), _p(status))
    return out, status


def root_condition(coeffs, roots) -> np.ndarray:
    a = _c128(coeffs)
    z = _c128(roots)
    n, K = a.shape
    kappa = np.zeros((n, K - 1))
    lib().or_root_condition(_p(a), n, K - 1, _p(z), _p(kappa))
    return kappa


def splat(roots, window, W: int = 256, H: int = 144, sigma: float = 1.5, scale: float = 1.0) -> np.ndarray:
    """Soft root density image [H, W] (float64) of the complex roots (any shape)."""
    z = _c128(roots).reshape(-1)
    img = np.zeros((H, W), np.float64)
    xmin, xmax, ymin, ymax = window
    lib().or_splat(_p(z), z.size, xmin, xmax, ymin, ymax, W, H, sigma, scale, _p(img))
    return img


def splat_grad(roots, G, window, W: int = 256, H: int = 144, sigma: float = 1.5, scale: float = 1.0) -> np.ndarray:
    """dL/dRe z + i dL/dIm z for every root (shape of roots) given G = dL/dimg [H, W]."""
    z = _c128(roots)
    flat = z.reshape(-1)
    g = np.ascontiguousarray(G, dtype=np.float64)
    assert g.shape == (H, W)
    out = np.zeros(flat.size, np.complex128)
    xmin, xmax, ymin, ymax = window
    lib().or_splat_grad(_p(flat), flat.size, xmin, xmax, ymin, ymax, W, H, sigma, scale, _p(g), _p(out))
    return out.reshape(z.shape)


def max_threads() -> int:
    return int(lib().or_max_threads())
