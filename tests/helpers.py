"""Shared test utilities: root-set matching and error metrics (no method arithmetic)."""
from __future__ import annotations

import numpy as np
from scipy.optimize import linear_sum_assignment


def match(a: np.ndarray, b: np.ndarray):
    """Optimal assignment between root sets a and b (1-D complex). Returns b reordered to a."""
    C = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(C)
    out = np.empty_like(b)
    out[r] = b[c]
    return out


def rel_err(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """|got - ref| / max(1, |ref|) elementwise."""
    return np.abs(got - ref) / np.maximum(1.0, np.abs(ref))


def matched_errors(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-root relative error [n, d] after matching each row of got to ref."""
    out = np.empty(got.shape, dtype=np.float64)
    for i in range(got.shape[0]):
        out[i] = rel_err(match(ref[i], got[i]), ref[i])
    return out


def matched(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """got with each row permuted to best match the same row of ref."""
    out = np.empty_like(got)
    for i in range(got.shape[0]):
        out[i] = match(ref[i], got[i])
    return out
