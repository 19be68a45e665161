"""The oracle pins catch plausible mistakes.

Each case copies oracle.c, plants one mistake of the kind a restatement of
the paper could contain (a dropped conjugate, a wrong sign or index, a
flipped orientation), builds the copy on the CPU and runs the pin tests
against it in a subprocess: at least one pin must fail. The untouched copy
must pass, so the failures come from the planted mistake.
"""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "givens_s_not_conjugated": ("*s = conj(b) / r;", "*s = b / r;"),
    "rotation_lower_sign": ("G[r * m + (r - 1)] = -conj(s);", "G[r * m + (r - 1)] = conj(s);"),
    "rotation_diagonal_not_conjugated": ("G[r * m + r] = conj(c);", "G[r * m + r] = c;"),
    "adjoint_not_conjugated_q": ("Y[j * m + i] = conj(X[i * m + j]);", "Y[j * m + i] = X[i * m + j];"),
    "matmul_transposed_operand": ("acc += X[i * m + k] * Y[k * m + j];", "acc += X[k * m + i] * Y[k * m + j];"),
    "q_accumulated_on_the_right": ("mat_mul(m, G, Qh, T); /* Q^H <- Q_r Q^H */",
                                   "mat_mul(m, Qh, G, T); /* Q^H <- Q_r Q^H */"),
    "rq_as_qr": ("mat_mul(m, B, Q, T); /* R Q */", "mat_mul(m, Q, B, T); /* R Q */"),
    "companion_sign": ("AT(A, n, i, n - 1) = -b[i];", "AT(A, n, i, n - 1) = b[i];"),
    "shift_not_restored": ("for (int i = 0; i < m; ++i) AT(A, n, i, i) += shift;", ""),
    "fixed_schedule_wrong_level": ("eig[m - 1] = AT(A, d, m - 1, m - 1);", "eig[m - 1] = AT(A, d, m - 2, m - 2);"),
    "wilkinson_far_root": ("cabs(mu_plus - d) <= cabs(mu_minus - d) ? mu_plus : mu_minus",
                           "cabs(mu_plus - d) > cabs(mu_minus - d) ? mu_plus : mu_minus"),
    "hist_rows_flipped": ("double fy = (ymax - y) * sy;", "double fy = (y - ymin) * sy;"),
    "legendre_weight": ("double wt = 2.0 / ((1.0 - t * t) * dp * dp);",
                        "double wt = 1.0 / ((1.0 - t * t) * dp * dp);"),
    "l2_rhs_not_conjugated": ("acc += wgt[pq] * ld(g + 2 * pq) * conj(pw[pq * K + j]);",
                              "acc += wgt[pq] * ld(g + 2 * pq) * pw[pq * K + j];"),
    "l2_missing_jacobian": ("wgt[p * nt + q] = wn[p] * rn[p] * (2.0 * M_PI / nt);",
                            "wgt[p * nt + q] = wn[p] * (2.0 * M_PI / nt);"),
    "adjoint_not_conjugated": ("g[k] += conj(-zk / dp) * gz;", "g[k] += (-zk / dp) * gz;"),
    "adjoint_derivative_index": ("dp = dp * z + (double)k * ld(a + 2 * k);",
                                 "dp = dp * z + (double)(k - 1) * ld(a + 2 * k);"),
    "splat_pixel_corner": ("const double du = u - (ix + 0.5);", "const double du = u - ix;"),
    "splat_sigma_factor": ("const double w = exp(-(du * du + dv * dv) / (2.0 * sigma * sigma)) - cut;",
                           "const double w = exp(-(du * du + dv * dv) / (sigma * sigma)) - cut;"),
    "splat_no_cut": ("const double w = exp(-(du * du + dv * dv) / (2.0 * sigma * sigma)) - cut;",
                     "const double w = exp(-(du * du + dv * dv) / (2.0 * sigma * sigma));"),
    "splat_rows_flipped": ("const double v = (ymax - roots[2 * j + 1]) / py;",
                           "const double v = (roots[2 * j + 1] - ymin) / py;"),
    "splat_grad_sign": ("gv += g * (-dv / (sigma * sigma)) * e;", "gv += g * (dv / (sigma * sigma)) * e;"),
    "splat_grad_scale": ("grad[2 * j] = scale * gu / px;", "grad[2 * j] = scale * gu * px;"),
    "splat_grad_y_orientation": ("grad[2 * j + 1] = -scale * gv / py;", "grad[2 * j + 1] = scale * gv / py;"),
}


def _build(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    hdr = tmp_path / "oracle.h"
    if not hdr.exists():
        hdr.write_text(open(os.path.join(ROOT, "oracle", "oracle.h")).read())
    so = tmp_path / f"{name}.so"
    sys.path.insert(0, ROOT)
    import oracle
    subprocess.run(["gcc", *oracle.CFLAGS, "-I", str(tmp_path), "-o", str(so), str(src), "-lm"], check=True)
    return str(so)


def _pins_pass(so: str) -> bool:
    env = dict(os.environ, ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode == 0


def test_unmutated_copy_passes(tmp_path):
    assert _pins_pass(_build(tmp_path, "clean", open(SRC).read()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    before, after = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(before) == 1, f"mutation site for {name} not found exactly once"
    assert not _pins_pass(_build(tmp_path, name, text.replace(before, after)))
