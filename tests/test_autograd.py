"""Adjoint backward under torch.autograd (FFTFunction / IFFTFunction).

Workload: loss = sum |W * FFT(x)|^2, x and W complex64 [65536, 1024], iid
standard normal (seed 2, x drawn first).  The backward of the forward FFT is
the unnormalised opposite-direction transform F^H, run by the library's own
kernel.  Checked against the FP64 oracle's gradient and against FP64 central
finite differences over every real coordinate of signals 0..63.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.helpers import FP32_TOL, max_rel_l2, rel_l2_per_signal, to_np

pytestmark = pytest.mark.gpu

import paper_2203_09384_gb300 as gb  # noqa: E402

N, BATCH, SUB = 1024, 65536, 64


@pytest.fixture(scope="module")
def workload():
    x, w = synth.normal_pair(BATCH, N, seed=2)
    return x, w


def fd_gradient(x_sub: np.ndarray, w_sub: np.ndarray, h: float = 1e-3) -> np.ndarray:
    """Central differences of each signal's own loss L_s = sum_k |W_k X_k|^2
    (FP64, oracle transform), for every real and imaginary coordinate."""
    n = x_sub.shape[1]
    grad = np.empty_like(x_sub)
    eye = np.eye(n)
    for s in range(x_sub.shape[0]):
        base = np.broadcast_to(x_sub[s], (n, n))
        rows = np.concatenate([base + h * eye, base - h * eye,
                               base + 1j * h * eye, base - 1j * h * eye])
        X = oracle.fft_radix2(rows, threads=8)
        L = np.sum(np.abs(w_sub[s][None, :] * X) ** 2, axis=1)
        d_re = (L[0:n] - L[n:2 * n]) / (2 * h)
        d_im = (L[2 * n:3 * n] - L[3 * n:4 * n]) / (2 * h)
        grad[s] = d_re + 1j * d_im
    return grad


def test_weighted_power_gradient(workload):
    x, w = workload
    xd = x.cuda().requires_grad_(True)
    wd = w.cuda()
    y = gb.FFTFunction.apply(xd)
    loss = (torch.abs(wd * y) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    g = xd.grad
    assert g is not None and g.dtype == torch.complex64 and g.shape == x.shape

    xs = x[:SUB].numpy().astype(np.complex128)
    ws = w[:SUB].numpy().astype(np.complex128)
    g_or, _ = oracle.grad_weighted_power(xs, ws, threads=8)
    g_fd = fd_gradient(xs, ws)
    # the oracle's gradient is pinned by the finite differences (quadratic loss)
    assert np.max(rel_l2_per_signal(g_or, g_fd)) < 1e-8
    got = to_np(g[:SUB])
    assert max_rel_l2(got, g_fd) <= FP32_TOL
    assert max_rel_l2(got, g_or) <= FP32_TOL
    # a seeded sample of the other signals against the oracle
    idx = torch.from_numpy(np.random.default_rng(2).choice(BATCH, 256, replace=False))
    g_or2, _ = oracle.grad_weighted_power(x[idx].numpy(), w[idx].numpy(), threads=8)
    assert max_rel_l2(to_np(g.index_select(0, idx.cuda())), g_or2) <= FP32_TOL


def test_backward_uses_the_adjoint_kernel():
    """The backward must run F^H (unnormalised inverse plan), not a torch op."""
    gb.clear_plan_cache()
    x = synth.normal(8, 256, seed=4).cuda().requires_grad_(True)
    y = gb.FFTFunction.apply(x)
    y.real.sum().backward()
    keys = {(k[1], k[2], k[3], k[4]) for k in gb._cache}
    assert (256, 8, True, False) in keys  # inverse, unnormalised
    # d/dx of sum(Re(F x)) with grad_output 1: F^H 1 = N * delta_0
    want = np.zeros((8, 256), np.complex128)
    want[:, 0] = 256
    assert np.max(np.abs(to_np(x.grad) - want)) <= 1e-4


@pytest.mark.parametrize("n", [2, 16, 64, 1024, 2048])
def test_adjoint_identity(n):
    """<F x, y> = <x, F^H y> for both autograd functions' backward maps."""
    x = synth.normal(33, n, seed=n).cuda()
    y = synth.normal(33, n, seed=n + 1).cuda()
    fx = gb.fft(x)
    fhy = gb.ifft(y, normalized=False)
    lhs = torch.vdot(fx.reshape(-1).to(torch.complex128), y.reshape(-1).to(torch.complex128))
    rhs = torch.vdot(x.reshape(-1).to(torch.complex128), fhy.reshape(-1).to(torch.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("n", [4, 128, 2048])
def test_inverse_function_gradient(n):
    """IFFTFunction: y = (1/N) F^H x, so dL/dx = (1/N) F g."""
    x = synth.normal(9, n, seed=3).cuda().requires_grad_(True)
    g = synth.normal(9, n, seed=5).cuda()
    y = gb.IFFTFunction.apply(x)
    (gx,) = torch.autograd.grad(y, x, grad_outputs=g)
    want = oracle.fft_radix2(g.cpu().numpy()) / n
    assert max_rel_l2(to_np(gx), want) <= FP32_TOL
    yo = oracle.fft_radix2(x.detach().cpu().numpy(), inverse=True)
    assert max_rel_l2(to_np(y), yo) <= FP32_TOL
