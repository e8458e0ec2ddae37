"""Shared test helpers: error metrics and GPU runs through the C-ABI."""
from __future__ import annotations

import os

import numpy as np
import torch

FP32_TOL = 1e-5  # per-signal relative L2 against the FP64 oracle


def rel_l2_per_signal(got, ref) -> np.ndarray:
    """||got - ref|| / ||ref|| per row (absolute error where ||ref|| == 0)."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    num = np.linalg.norm(got - ref, axis=-1)
    den = np.linalg.norm(ref, axis=-1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def max_rel_l2(got, ref) -> float:
    e = rel_l2_per_signal(got, ref)
    return float(e.max()) if e.size else 0.0


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.complex128)


def c32_encode(x) -> tuple[torch.Tensor, torch.Tensor]:
    """complex32 storage of complex values [batch, n]: binary16 (re, im) pairs
    and one int8 exponent per signal, value = stored * 2^exp, the exponent
    putting the signal's largest component in [2^14, 2^15).  Returns CPU
    tensors (torch.complex32 [batch, n], torch.int8 [batch])."""
    z = np.asarray(x, dtype=np.complex128)
    m = np.maximum(np.abs(z.real), np.abs(z.imag)).max(axis=1)
    e = np.where(m > 0, np.frexp(m)[1] - 15, 0).astype(np.int64)
    pairs = np.stack([z.real, z.imag], axis=-1) * np.ldexp(1.0, -e)[:, None, None]
    h = torch.from_numpy(pairs.astype(np.float16).reshape(z.shape[0], -1).copy())
    return h.view(torch.complex32), torch.from_numpy(e.astype(np.int8))


def c32_decode(stored: torch.Tensor, exp: torch.Tensor) -> np.ndarray:
    """Inverse of c32_encode (exact): complex128 [batch, n]."""
    h = stored.detach().contiguous().view(torch.float16).cpu().numpy().astype(np.float64)
    h = h.reshape(stored.shape[0], -1, 2)
    e = exp.detach().cpu().numpy().astype(np.int64)
    return (h[..., 0] + 1j * h[..., 1]) * np.ldexp(1.0, e)[:, None]


def c32_max_stored(stored: torch.Tensor) -> np.ndarray:
    """Largest |component| of each signal as stored (before the exponent)."""
    h = stored.detach().contiguous().view(torch.float16).cpu().numpy().astype(np.float64)
    return np.abs(h.reshape(stored.shape[0], -1)).max(axis=1)


def c32_to(x: torch.Tensor, device) -> torch.Tensor:
    """Move a complex32 tensor (through its binary16 view)."""
    return x.contiguous().view(torch.float16).to(device).view(torch.complex32)


def every_signal_violations(x: torch.Tensor, y: torch.Tensor, tol: float,
                            chunk_elems: int = 1 << 24) -> torch.Tensor:
    """Check every signal of a forward transform y = F x (device tensors
    [batch, n], any complex dtype) against three consequences of the parity
    bar ||y - X|| <= tol ||X|| (X the exact DFT; absolute tol where X = 0):

    * Parseval, ||X|| = sqrt(N) ||x||, so | ||y|| - sqrt(N) ||x|| | <= bound;
    * bin 0 of Eq. (dft) is the plain sum of x: |y_0 - sum x| <= bound;
    * bin N/2 is the alternating sum: |y_{N/2} - sum (-1)^n x_n| <= bound
      (any one component's error is at most the L2 norm of the error).

    Sums run in FP64 on the device, from the input alone, a chunk of rows at a
    time.  Returns the indices of the signals that break any of them."""
    batch, n = x.shape
    sign = torch.ones(n, dtype=torch.float64, device=x.device)
    sign[1::2] = -1.0
    rows = max(1, chunk_elems // n)
    bad = []
    for r0 in range(0, batch, rows):
        xd = x[r0:r0 + rows].to(torch.complex128)
        yd = y[r0:r0 + rows].to(torch.complex128)
        ref_norm = torch.linalg.vector_norm(xd, dim=1) * (n ** 0.5)
        bound = torch.where(ref_norm > 0, tol * ref_norm, torch.full_like(ref_norm, tol))
        bound = bound * (1 + 1e-9) + 1e-300  # FP64 summation slack
        ok = (torch.linalg.vector_norm(yd, dim=1) - ref_norm).abs() <= bound
        ok &= (yd[:, 0] - xd.sum(dim=1)).abs() <= bound
        if n >= 2:
            ok &= (yd[:, n // 2] - (xd * sign).sum(dim=1)).abs() <= bound
        bad.append(torch.nonzero(~ok).flatten() + r0)
        del xd, yd
    return torch.cat(bad).cpu() if bad else torch.empty(0, dtype=torch.int64)


def oracle_max_rel_l2(x: torch.Tensor, y: torch.Tensor, inverse: bool = False, normalized: bool = True,
                      rows=None, chunk_elems: int = 1 << 24, threads: int | None = None):
    """Compare signals of y (a device or host tensor [batch, n], the library's
    transform of x) element by element with the FP64 oracle's transform of
    the same FP32 inputs, a chunk of signals at a time so host memory stays
    bounded.  ``rows`` selects the signals (an index array; None = every
    signal of the batch).  Returns (largest per-signal relative L2 error,
    index of the signal that has it)."""
    import oracle

    batch, n = x.shape
    threads = threads or os.cpu_count() or 1
    step = max(1, chunk_elems // n)
    worst, where = 0.0, -1
    if rows is None:
        chunks = ((r0, None) for r0 in range(0, batch, step))
    else:
        rows = np.asarray(rows, dtype=np.int64)
        chunks = ((k, rows[k:k + step]) for k in range(0, rows.size, step))
    for k, idx in chunks:
        if idx is None:
            xs, ys, base = x[k:k + step], y[k:k + step], np.arange(k, min(k + step, batch))
        else:
            ti = torch.from_numpy(idx).to(x.device)
            xs, ys, base = x.index_select(0, ti), y.index_select(0, ti.to(y.device)), idx
        want = oracle.reference(xs.cpu().numpy(), inverse, normalized, threads=threads)
        e = rel_l2_per_signal(ys.cpu().numpy(), want)
        i = int(e.argmax())
        if e[i] > worst:
            worst, where = float(e[i]), int(base[i])
    return worst, where
