"""gbfft: batched 1-D C2C power-of-two FFT on GB300 (sm_103a).

Python face of the C-ABI in ``include/gbfft.h`` (libgbfft.so, built in-tree).
PyTorch supplies device memory and streams; every transform runs in the
library's own CUDA kernels.  There is no CPU or library fallback: without the
built extension, calls raise.

    import paper_2203_09384_gb300 as gbfft
    X = gbfft.fft(x)                 # x: complex64 CUDA tensor [..., N]
    x2 = gbfft.ifft(X)               # Eq. (idft): includes 1/N
    y = gbfft.FFTFunction.apply(x)   # differentiable (adjoint backward)
"""
from __future__ import annotations

import collections
import threading

import torch

from ._abi import (FFT_C32, FFT_C64, FFT_C64_TC_BF16, FFT_C64_TC_F16, FFT_FLAG_SCALE_FORWARD,  # noqa: F401
                   fft_execute_c32,
                   FFT_FLAG_UNNORMALIZED, FFT_FLAG_VARIANT, fft_get_default_variant,
                   fft_plan_create_ragged, fft_ragged_variant_count, fft_variant_dtype,
                   DTYPE_NAMES,
                   fft_set_default_variant, fft_variant_count,
                   FFT_FORWARD, FFT_INVERSE, FFTError, STATUS, fft_execute, fft_plan_create,
                   fft_plan_create_ex, fft_plan_destroy, fft_plan_get_error, fft_plan_get_info,
                   fft_plan_set_wait_limit, FFT_FLAG_TEST_STALL, FFT_FLAG_HOST_STAGING,
                   fft_execute_host,
                   fft_validate, lib, fft_set_default_ragged_variant, fft_get_default_ragged_variant)
from . import autotune  # noqa: E402

__all__ = ["Plan", "RaggedPlan", "fft", "ifft", "FFTFunction", "IFFTFunction", "fft_plan_create",
           "fft_plan_create_ex", "fft_plan_create_ragged", "fft_execute", "fft_plan_destroy",
           "fft_plan_get_error", "FFTError", "lib"]

_DTYPES = {"c64": FFT_C64, "tc_f16": FFT_C64_TC_F16, "tc_bf16": FFT_C64_TC_BF16, "c32": FFT_C32}


def _cuda_device(device) -> torch.device:
    """The plan's device with an explicit index ("cuda" means the current one)."""
    d = torch.device(device) if device is not None else torch.device("cuda")
    if d.type != "cuda":
        raise ValueError(f"plans live on a CUDA device, got {d}")
    return d if d.index is not None else torch.device("cuda", torch.cuda.current_device())


def _check_buffer(t: torch.Tensor, name: str, dtype, device, numel: int, at_least: bool = False) -> None:
    """A buffer handed to the C-ABI as a bare pointer: the library cannot see
    its size, dtype or device, so they are checked here before the launch."""
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if (t.numel() < numel) if at_least else (t.numel() != numel):
        raise ValueError(f"{name} has {t.numel()} elements, needs {'at least ' if at_least else ''}{numel}")


class Plan:
    """One planned transform: length ``n``, ``batch`` signals, a direction.

    ``normalized=False`` with ``inverse=True`` drops the 1/N (the adjoint F^H);
    ``normalized=True`` with ``inverse=False`` is the plain Eq. (dft), and
    ``scale_forward=True`` multiplies a forward transform by 1/N.
    """

    def __init__(self, n: int, batch: int, inverse: bool = False, dtype: str = "c64",
                 normalized: bool = True, device=None, scale_forward: bool = False,
                 variant: int | None = None, extra_flags: int = 0, host_staging: bool = False):
        self.n, self.batch, self.inverse = int(n), int(batch), bool(inverse)
        self.dtype = dtype
        self.normalized = normalized
        self.device = _cuda_device(device)
        flags = 0 if normalized else FFT_FLAG_UNNORMALIZED
        if scale_forward and not inverse:
            flags |= FFT_FLAG_SCALE_FORWARD
        if variant is not None:
            flags |= FFT_FLAG_VARIANT(variant)
        flags |= int(extra_flags)
        if host_staging:
            flags |= FFT_FLAG_HOST_STAGING
        direction = FFT_INVERSE if inverse else FFT_FORWARD
        self.handle = None
        with torch.cuda.device(self.device):
            autotune.autoload(self.device)
            self.handle = fft_plan_create_ex(self.n, self.batch, direction, _DTYPES[dtype], flags)

    def info(self):
        return fft_plan_get_info(self.handle)

    def execute(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        _check_buffer(x, "x", torch.complex64, self.device, self.n * self.batch)
        if out is None:
            out = torch.empty_like(x)
        else:
            _check_buffer(out, "out", torch.complex64, self.device, self.n * self.batch)
        with torch.cuda.device(x.device):
            s = stream if stream is not None else torch.cuda.current_stream(x.device)
            fft_execute(self.handle, x.data_ptr(), out.data_ptr(), s.cuda_stream)
        return out

    def execute_c32(self, x: torch.Tensor, x_exp: torch.Tensor, out: torch.Tensor | None = None,
                    out_exp: torch.Tensor | None = None, stream=None):
        """complex32 storage (plan dtype "c32"): x is a torch.complex32 CUDA
        tensor, x_exp an int8 tensor of one exponent per signal (value =
        stored * 2^exp).  Returns (out, out_exp) in the same representation."""
        _check_buffer(x, "x", torch.complex32, self.device, self.n * self.batch)
        _check_buffer(x_exp, "x_exp", torch.int8, self.device, self.batch)
        if out is None:
            out = torch.empty_like(x)
        else:
            _check_buffer(out, "out", torch.complex32, self.device, self.n * self.batch)
        if out_exp is None:
            out_exp = torch.empty(self.batch, dtype=torch.int8, device=x.device)
        else:
            _check_buffer(out_exp, "out_exp", torch.int8, self.device, self.batch)
        with torch.cuda.device(x.device):
            s = stream if stream is not None else torch.cuda.current_stream(x.device)
            fft_execute_c32(self.handle, x.data_ptr(), x_exp.data_ptr(), out.data_ptr(),
                            out_exp.data_ptr(), s.cuda_stream)
        return out, out_exp

    def execute_host(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Transform a host (CPU, ideally pinned) tensor through the plan's
        chunked copy/transform/copy pipeline; synchronises the stream."""
        cpu = torch.device("cpu")
        _check_buffer(x, "x", torch.complex64, cpu, self.n * self.batch)
        if out is None:
            out = torch.empty(x.shape, dtype=x.dtype, pin_memory=x.is_pinned())
        else:
            _check_buffer(out, "out", torch.complex64, cpu, self.n * self.batch)
        with torch.cuda.device(self.device):
            s = stream if stream is not None else torch.cuda.current_stream(self.device)
            fft_execute_host(self.handle, x.data_ptr(), out.data_ptr(), s.cuda_stream)
            s.synchronize()
        return out

    def error(self) -> int:
        return fft_plan_get_error(self.handle)

    def set_wait_limit(self, nanoseconds: int) -> None:
        fft_plan_set_wait_limit(self.handle, nanoseconds)

    def close(self):
        if self.handle:
            fft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RaggedPlan:
    """Mixed-length batch: signal i occupies elements [offsets[i], offsets[i+1])
    of a flat complex64 buffer; one persistent launch transforms them all."""

    def __init__(self, offsets, inverse: bool = False, normalized: bool = True,
                 scale_forward: bool = False, variant: int | None = None, device=None,
                 extra_flags: int = 0):
        offs = [int(v) for v in (offsets.tolist() if hasattr(offsets, "tolist") else offsets)]
        if len(offs) < 1:
            raise ValueError("offsets needs count + 1 entries")
        self.offsets = offs
        self.count = len(offs) - 1
        self.total = offs[-1]
        self.inverse = inverse
        self.device = _cuda_device(device)
        flags = 0 if normalized else FFT_FLAG_UNNORMALIZED
        if scale_forward and not inverse:
            flags |= FFT_FLAG_SCALE_FORWARD
        if variant is not None:
            flags |= FFT_FLAG_VARIANT(variant)
        flags |= int(extra_flags)
        self.handle = None
        with torch.cuda.device(self.device):
            autotune.autoload(self.device)
            self.handle = fft_plan_create_ragged(offs, FFT_INVERSE if inverse else FFT_FORWARD,
                                                 FFT_C64, flags)

    def info(self):
        return fft_plan_get_info(self.handle)

    def execute(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        _check_buffer(x, "x", torch.complex64, self.device, self.total, at_least=True)
        if out is None:
            out = torch.empty_like(x)
        else:
            _check_buffer(out, "out", torch.complex64, self.device, self.total, at_least=True)
        with torch.cuda.device(x.device):
            s = stream if stream is not None else torch.cuda.current_stream(x.device)
            fft_execute(self.handle, x.data_ptr(), out.data_ptr(), s.cuda_stream)
        return out

    def capture(self, x: torch.Tensor, out: torch.Tensor) -> "torch.cuda.CUDAGraph":
        """Capture execute(x, out) in a CUDA graph (the persistent kernel, after a
        work-counter reset for the variants that use a counter)."""
        s = torch.cuda.Stream(device=x.device)
        s.wait_stream(torch.cuda.current_stream(x.device))
        with torch.cuda.stream(s):
            self.execute(x, out)  # warm-up outside the capture
        torch.cuda.current_stream(x.device).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.execute(x, out)
        return g

    def error(self) -> int:
        return fft_plan_get_error(self.handle)

    def set_wait_limit(self, nanoseconds: int) -> None:
        fft_plan_set_wait_limit(self.handle, nanoseconds)

    def close(self):
        if self.handle:
            fft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Plans made by fft / ifft / the autograd functions, least recently used
# first.  Each holds a device allocation, so the cache is bounded: a workload
# of ever new shapes (say, autograd over varying batch sizes) keeps at most
# PLAN_CACHE_SIZE plans alive.
PLAN_CACHE_SIZE = 64
_cache: "collections.OrderedDict" = collections.OrderedDict()
_cache_lock = threading.Lock()


def _retire(p: Plan) -> None:
    """Destroy an evicted plan once no kernel of it can still be running."""
    torch.cuda.synchronize(p.device)
    p.close()


def get_plan(n: int, batch: int, inverse: bool, normalized: bool, device, dtype: str = "c64",
             scale_forward: bool = False) -> Plan:
    key = (str(device), n, batch, inverse, normalized, dtype, scale_forward)
    with _cache_lock:
        p = _cache.get(key)
        if p is not None:
            _cache.move_to_end(key)
            return p
        p = Plan(n, batch, inverse, dtype, normalized, device, scale_forward)
        _cache[key] = p
        while len(_cache) > PLAN_CACHE_SIZE:
            _, old = _cache.popitem(last=False)
            _retire(old)
        return p


def clear_plan_cache():
    with _cache_lock:
        plans = list(_cache.values())
        _cache.clear()
    for p in plans:
        _retire(p)


def _run(x: torch.Tensor, inverse: bool, normalized: bool = True, dtype: str = "c64",
         scale_forward: bool = False) -> torch.Tensor:
    if x.dtype != torch.complex64:
        raise TypeError("gbfft works on complex64 tensors")
    if not x.is_cuda:
        raise TypeError("gbfft works on CUDA tensors")
    n = x.shape[-1]
    x = x.contiguous()
    batch = x.numel() // n if n > 0 else 0
    plan = get_plan(n, batch, inverse, normalized, x.device, dtype, scale_forward)
    return plan.execute(x)


def fft(x: torch.Tensor, dtype: str = "c64") -> torch.Tensor:
    """Forward DFT (Eq. (dft)) along the last dimension."""
    return _run(x, False, True, dtype)


def ifft(x: torch.Tensor, normalized: bool = True, dtype: str = "c64") -> torch.Tensor:
    """Inverse DFT (Eq. (idft)) along the last dimension; 1/N unless normalized=False."""
    return _run(x, True, normalized, dtype)


class FFTFunction(torch.autograd.Function):
    """Differentiable forward FFT.  Backward applies the adjoint F^H, i.e. the
    unnormalised opposite-direction transform, in the library's kernel."""

    @staticmethod
    def forward(ctx, x):
        return _run(x, inverse=False)

    @staticmethod
    def backward(ctx, g):
        return _run(g.contiguous(), inverse=True, normalized=False)


class IFFTFunction(torch.autograd.Function):
    """Differentiable normalised inverse FFT; backward is (1/N) F g."""

    @staticmethod
    def forward(ctx, x):
        return _run(x, inverse=True)

    @staticmethod
    def backward(ctx, g):
        return _run(g.contiguous(), inverse=False, scale_forward=True)
