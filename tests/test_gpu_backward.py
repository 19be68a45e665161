"""GPU parity of the implicit-differentiation adjoint and the autograd Function."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2507_02164_gb300 import api, workloads as WL
from tests.gpu_common import require_gpu, roots_poly_major, to_soa
from tests.helpers import match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


@pytest.mark.parametrize("dtype,rtol", [(torch.complex128, 1e-12), (torch.complex64, 1e-4)])
def test_backward_matches_oracle_adjoint(dev, orc, dtype, rtol):
    n = 4096 + 5
    co = WL.gaussian(4, n, 6)
    if dtype == torch.complex64:
        co = co.astype(np.complex64).astype(np.complex128)
    roots, _, _, _ = orc.solve(co)
    g = np.random.default_rng(3)
    gz = g.standard_normal(roots.shape) + 1j * g.standard_normal(roots.shape)
    ref, ref_st = orc.roots_backward(co, roots, gz)
    coeffs_t = to_soa(co, dev, dtype)
    roots_t = to_soa(roots, dev)
    gz_t = to_soa(gz, dev)
    status = torch.empty(n, dtype=torch.uint8, device=dev)
    got = api.roots_backward(coeffs_t, roots_t, gz_t, status=status)
    torch.cuda.synchronize()
    got = got.cpu().numpy().T.astype(np.complex128)
    scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-300)
    assert (np.abs(got - ref) / scale).max() <= rtol
    assert np.array_equal(status.cpu().numpy(), ref_st)


def test_backward_singular_root_sets_status(dev):
    co = np.array([[1.0, -2.0, 1.0], [2.0, -3.0, 1.0]], dtype=complex)  # (z-1)^2 ; (z-1)(z-2)
    z = np.array([[1.0, 1.0], [1.0, 2.0]], dtype=complex)
    status = torch.empty(2, dtype=torch.uint8, device=dev)
    got = api.roots_backward(to_soa(co, dev), to_soa(z, dev), to_soa(np.ones_like(z), dev), status=status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [2, 0]
    assert np.all(got.cpu().numpy()[:, 0] == 0)


def test_autograd_function_matches_finite_differences(dev, orc):
    """L = sum_i sum_j |z_ij|^2 w_ij; central differences (h = 1e-6, FP64,
    oracle re-solves rematched to the unperturbed roots) on 64 polynomials."""
    n = 64
    co = WL.gaussian(4, n, 6)
    wts = np.random.default_rng(1).uniform(0.5, 1.5, (n, 6))
    coeffs_t = to_soa(co, dev).requires_grad_(True)
    roots_t, _ = api.roots(coeffs_t, "plain")
    w_t = torch.from_numpy(np.ascontiguousarray(wts.T)).to(dev)
    loss = (w_t * roots_t.abs() ** 2).sum()
    loss.backward()
    grad = coeffs_t.grad.cpu().numpy().T
    z0 = roots_poly_major(roots_t.detach())

    def L(c, i):
        r, _, _, _ = orc.solve(c[None, :])
        r = match(z0[i], r[0])
        return float((wts[i] * np.abs(r) ** 2).sum())

    h = 1e-6
    checked = 0
    for i in range(n):
        sep = np.min(np.abs(z0[i][:, None] - z0[i][None, :]) + 1e9 * np.eye(6))
        if sep < 1e-2:
            continue
        fd = np.zeros(7, complex)
        for k in range(7):
            for unit in (1.0, 1j):
                cp = co[i].copy()
                cp[k] += h * unit
                cm = co[i].copy()
                cm[k] -= h * unit
                fd[k] += unit * (L(cp, i) - L(cm, i)) / (2 * h)
        rel = np.abs(fd - grad[i]) / max(1.0, np.abs(grad[i]).max())
        assert rel.max() <= 1e-6, (i, rel)
        checked += 1
    assert checked > 40


def test_soft_density_loss_gradients_on_1024_polynomials(dev, orc):
    """The differentiation configuration: L = sum |z|^2 + sum (D - T)^2 with
    D the Gaussian splat (256 x 144) of the roots of 1,024 complex-Gaussian
    degree-6 polynomials and T the splat of a second seeded batch (2^16
    polynomials). The gradient through RootsFn (GPU solve + adjoint kernel)
    equals the oracle's implicit gradient to 1e-12 and central finite
    differences (h = 1e-6, FP64, oracle re-solves and the oracle's image,
    rematched) to 1e-6 for every polynomial whose roots are separated by
    more than 1e-2. The image and its pull-back run in the CUDA splat
    kernels."""
    from paper_2507_02164_gb300 import splat as SP
    n = 1024
    co = WL.gaussian(4, n, 6)
    tgt, _, _, _ = orc.solve(WL.gaussian(5, 1 << 16, 6))
    T = torch.from_numpy(orc.splat(tgt, SP.WINDOW, scale=1.0 / tgt.size))
    coeffs_t = to_soa(co, dev).requires_grad_(True)
    roots_t, status = api.roots(coeffs_t, "plain")
    L = SP.loss(roots_t, T.to(dev))
    gz, = torch.autograd.grad(L, roots_t, retain_graph=True)
    L.backward()
    grad = coeffs_t.grad.cpu().numpy().T
    z0 = roots_poly_major(roots_t.detach())
    # the oracle's adjoint with the same dL/dz
    g_or, st_or = orc.roots_backward(co, z0, gz.cpu().numpy().T)
    assert np.all(st_or == 0)
    scale = np.abs(g_or).max(axis=1, keepdims=True)
    assert (np.abs(grad - g_or) / scale).max() <= 1e-12
    # finite differences of the loss change caused by one polynomial
    N_roots = 6 * n
    D0 = orc.splat(z0, SP.WINDOW, scale=1.0 / N_roots)
    R0 = D0 - T.numpy()

    def dloss(i, zi_new):
        zi_old = z0[i]
        dD = orc.splat(zi_new, SP.WINDOW, scale=1.0 / N_roots) - orc.splat(zi_old, SP.WINDOW, scale=1.0 / N_roots)
        return float((np.abs(zi_new) ** 2).sum() - (np.abs(zi_old) ** 2).sum() + (dD * (2 * R0 + dD)).sum())

    h = 1e-6
    checked = 0
    for i in range(n):
        sep = np.min(np.abs(z0[i][:, None] - z0[i][None, :]) + 1e9 * np.eye(6))
        if sep < 1e-2:
            continue
        fd = np.zeros(7, complex)
        for k in range(7):
            for unit in (1.0, 1j):
                cp = co[i].copy()
                cp[k] += h * unit
                cm = co[i].copy()
                cm[k] -= h * unit
                rp, _, _, _ = orc.solve(cp[None, :])
                rm, _, _, _ = orc.solve(cm[None, :])
                rp = match(z0[i], rp[0])
                rm = match(z0[i], rm[0])
                fd[k] += unit * (dloss(i, rp) - dloss(i, rm)) / (2 * h)
        rel = np.abs(fd - grad[i]) / max(1.0, np.abs(grad[i]).max())
        assert rel.max() <= 1e-6, (i, rel.max())
        checked += 1
    assert checked > 900


def test_full_size_adjoint_sampled(dev, orc):
    """2^20 degree-6 polynomials (complex128): forward mixed roots, adjoint of
    L = sum |z|^2; 4096 sampled polynomials match the oracle's adjoint of the
    same roots to 1e-12."""
    n = 1 << 20
    co = WL.gaussian(4, n, 6)
    coeffs = to_soa(co, dev)
    roots, status = api.roots_batched(coeffs, mode="mixed")
    grad = api.roots_backward(coeffs, roots, 2.0 * roots)
    torch.cuda.synchronize()
    idx = np.linspace(0, n - 1, 4096).astype(np.int64)
    z = roots.cpu().numpy().T[idx]
    g_ref, st = orc.roots_backward(co[idx], z, 2.0 * z)
    g = grad.cpu().numpy().T[idx]
    ok = st == 0
    scale = np.maximum(np.abs(g_ref).max(axis=1, keepdims=True), 1e-300)
    assert (np.abs(g - g_ref)[ok] / scale[ok]).max() <= 1e-12
