"""Seeded synthetic inputs for the batched C2C FFT workloads.

This module holds no transform arithmetic: it only draws numbers.  It is the
one module that both the oracle-side tests and the CUDA-side tests/benchmark
use, so both see exactly the same complex64 values.

All CPU draws use ``torch.Generator().manual_seed(seed)`` (deterministic across
machines and PyTorch versions we run on).  Shapes are ``[batch, n]`` complex64,
signal-contiguous (batch stride n), the layout the library consumes.

Workloads (each one is what the paper or the benchmark definition describes):
  * ``uniform``   - re/im iid U[-1, 1]                       (batched sweeps)
  * ``normal``    - re/im iid N(0, 1)                        (gradient loss)
  * ``ramp``      - x_n = n, the paper's test input f(x) = x (Sec. 6)
  * ``ragged_lengths`` - log2 N uniform over {lo..hi}        (mixed lengths)
  * ``scaled_normal``  - N(0,1) signals scaled by 10^U(-3,3) per signal
"""
from __future__ import annotations

import torch


def _gen(seed: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def uniform(batch: int, n: int, seed: int, device="cpu") -> torch.Tensor:
    """complex64 [batch, n], re and im iid uniform on [-1, 1]."""
    g = _gen(seed, device)
    r = torch.rand(batch, n, 2, generator=g, device=device, dtype=torch.float32)
    r.mul_(2.0).sub_(1.0)
    return torch.view_as_complex(r)


def normal(batch: int, n: int, seed: int, device="cpu", generator=None) -> torch.Tensor:
    """complex64 [batch, n], re and im iid standard normal."""
    g = generator if generator is not None else _gen(seed, device)
    r = torch.randn(batch, n, 2, generator=g, device=device, dtype=torch.float32)
    return torch.view_as_complex(r)


def normal_pair(batch: int, n: int, seed: int, device="cpu"):
    """(x, W) drawn in that order from one generator, both complex N(0,1)."""
    g = _gen(seed, device)
    x = normal(batch, n, seed, device, generator=g)
    w = normal(batch, n, seed, device, generator=g)
    return x, w


def ramp(n: int, batch: int = 1) -> torch.Tensor:
    """complex64 [batch, n] with x_k = k (imaginary part 0)."""
    r = torch.arange(n, dtype=torch.float32).repeat(batch, 1)
    return torch.complex(r, torch.zeros_like(r))


def ragged_lengths(count: int, seed: int, lo_log2: int = 4, hi_log2: int = 11):
    """int64 tensor of lengths 2^u, u uniform over the integers lo..hi."""
    g = _gen(seed)
    u = torch.randint(lo_log2, hi_log2 + 1, (count,), generator=g, dtype=torch.int64)
    return torch.pow(2, u)


def ragged_offsets(lengths: torch.Tensor) -> torch.Tensor:
    """Exclusive prefix sum with the total appended: offsets[count] = sum(lengths)."""
    off = torch.zeros(lengths.numel() + 1, dtype=torch.int64)
    off[1:] = torch.cumsum(lengths.to(torch.int64), 0)
    return off


def ragged_uniform(lengths: torch.Tensor, seed: int) -> torch.Tensor:
    """Flat complex64 buffer of sum(lengths) elements, re/im iid U[-1, 1]."""
    total = int(lengths.sum())
    return uniform(1, total, seed).reshape(total)


def scaled_normal(batch: int, n: int, seed: int, lo: float = -3.0, hi: float = 3.0, device="cpu"):
    """complex64 [batch, n]: N(0,1) signals, signal i scaled by 10^u_i, u_i ~ U(lo, hi).

    The signal values are drawn first, then the exponents, from one generator.
    Returns (x, scale) with scale a float64 tensor [batch] (on the CPU).
    """
    g = _gen(seed, device)
    x = normal(batch, n, seed, device=device, generator=g)
    u = torch.rand(batch, generator=g, dtype=torch.float64, device=device) * (hi - lo) + lo
    s = torch.pow(torch.tensor(10.0, dtype=torch.float64, device=device), u)
    xs = torch.view_as_complex(torch.view_as_real(x) * s.to(torch.float32)[:, None, None])
    return xs, s.cpu()


def delta(n: int, pos: int = 0, batch: int = 1) -> torch.Tensor:
    x = torch.zeros(batch, n, dtype=torch.complex64)
    x[:, pos] = 1.0
    return x
