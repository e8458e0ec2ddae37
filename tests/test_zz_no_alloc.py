"""fft_execute_noalloc: the transform for callers that cannot allocate device
memory (for example a process whose caching allocator owns all free device
memory, or code that must not take the device-wide stall cudaMalloc/cudaFree
can cause).  Its scratch is a static device array shared by all calls, so
these checks run two calls in a row, with different lengths in between, and
compare each result with the planned path (fft_plan_create + fft_execute):
bit for bit, since both generate the same FP32 twiddle table by the same
steps and run the same kernel, and with the FP64 oracle within the FP32
tolerance.

This file is named to be collected last; it also passes on its own in a fresh
process (``pytest tests/test_zz_no_alloc.py -m gpu``).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.helpers import FP32_TOL, max_rel_l2, to_np

pytestmark = pytest.mark.gpu

import paper_2203_09384_gb300 as gb  # noqa: E402
from paper_2203_09384_gb300 import _abi  # noqa: E402

CASES = [
    # (n, batch, direction, flags)
    (2048, 3001, _abi.FFT_FORWARD, 0),
    (64, 777, _abi.FFT_INVERSE, 0),
    (1024, 4099, _abi.FFT_INVERSE, _abi.FFT_FLAG_UNNORMALIZED),
    (8, 10007, _abi.FFT_FORWARD, 0),
    (512, 1500, _abi.FFT_FORWARD, _abi.FFT_FLAG_SCALE_FORWARD),
    (32, 513, _abi.FFT_INVERSE, 0),
    (2, 1, _abi.FFT_FORWARD, 0),
]


def planned(x, n, batch, direction, flags):
    out = torch.empty_like(x)
    h = _abi.fft_plan_create_ex(n, batch, direction, _abi.FFT_C64, flags)
    try:
        _abi.fft_execute(h, x.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    finally:
        _abi.fft_plan_destroy(h)
    return out


def noalloc(x, n, batch, direction, flags):
    out = torch.full_like(x, float("nan"))
    _abi.fft_execute_noalloc(n, batch, direction, flags, x.data_ptr(), out.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    return out


def test_matches_planned_path_on_two_calls_in_a_row():
    inputs = {c: synth.uniform(c[1], c[0], seed=31 + i).cuda() for i, c in enumerate(CASES)}
    refs = {c: planned(inputs[c], *c) for c in CASES}
    for c in CASES:  # consecutive calls alternate lengths, so the array is rewritten each time
        first = noalloc(inputs[c], *c)
        second = noalloc(inputs[c], *c)
        torch.cuda.synchronize()
        n, batch, direction, flags = c
        inverse = direction == _abi.FFT_INVERSE
        normalized = not (flags & _abi.FFT_FLAG_UNNORMALIZED)
        want = oracle.reference(inputs[c].cpu().numpy(), inverse, normalized, threads=8)
        if flags & _abi.FFT_FLAG_SCALE_FORWARD:
            want = want / n
        for got in (first, second):
            assert torch.equal(got, refs[c]), c  # bit for bit
            err = max_rel_l2(to_np(got), want)
            assert err <= FP32_TOL, (c, err)


def _fp32_variants():
    return [(n, v) for n in [2 ** k for k in range(1, 12)] for v in range(_abi.fft_variant_count(n))
            if _abi.fft_variant_dtype(n, v) == _abi.FFT_C64]


@pytest.mark.parametrize("n,variant", _fp32_variants())
def test_every_fp32_schedule_bit_identical_to_planned(n, variant):
    """Every compiled FP32 schedule through FFT_FLAG_VARIANT(k): its twiddle
    table (written into the static array by this call) and its result equal
    the planned path's bit for bit, forward and inverse, twice in a row."""
    batch = 3 * 152 + 5
    x = synth.uniform(batch, n, seed=50 + variant).cuda()
    flags = _abi.FFT_FLAG_VARIANT(variant)
    for direction in (_abi.FFT_FORWARD, _abi.FFT_INVERSE):
        ref = planned(x, n, batch, direction, flags)
        for _ in range(2):
            got = noalloc(x, n, batch, direction, flags)
            torch.cuda.synchronize()
            assert torch.equal(got, ref), (n, variant, direction)


def test_allocates_no_device_memory():
    n, batch = 1024, 8192
    x = synth.uniform(batch, n, seed=5).cuda()
    out = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    lengths = (2, 16, 256, 2048, 1024)

    def sweep():
        for k in lengths:
            _abi.fft_execute_noalloc(k, (n * batch) // k, 1, 0, x.data_ptr(), out.data_ptr(), s)
        torch.cuda.synchronize()

    sweep()  # set-up calls; the CUDA driver also loads each kernel's code on first launch
    free_before, _ = torch.cuda.mem_get_info()
    sweep()
    sweep()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_rejects_bad_requests():
    x = torch.zeros(64, dtype=torch.complex64, device="cuda")
    L = _abi.lib()
    code = _abi.STATUS_CODE
    p = x.data_ptr()
    assert L.fft_execute_noalloc(12, 1, 0, 0, p, p, None) == code["FFT_ERR_INVALID_SIZE"]
    assert L.fft_execute_noalloc(4096, 1, 0, 0, p, p, None) == code["FFT_ERR_INVALID_SIZE"]
    assert L.fft_execute_noalloc(8, 1, 0, 0, p + 8, p + 8, None) == code["FFT_ERR_MISALIGNED"]
    assert L.fft_execute_noalloc(8, 4, 0, 0, p, p + 16, None) == code["FFT_ERR_OVERLAP"]
    assert L.fft_execute_noalloc(8, 1, 0, _abi.FFT_FLAG_VARIANT(7), p, p, None) == \
        code["FFT_ERR_INVALID_VALUE"]
    # flags this call does not honour are refused, not ignored
    for bad in (_abi.FFT_FLAG_TEST_STALL, _abi.FFT_FLAG_HOST_STAGING, 1 << 5):
        assert L.fft_execute_noalloc(8, 1, 0, bad, p, p, None) == code["FFT_ERR_INVALID_VALUE"]
    tc = next(v for v in range(_abi.fft_variant_count(256))
              if _abi.fft_variant_dtype(256, v) != _abi.FFT_C64)  # a tensor-core or complex32 schedule
    assert L.fft_execute_noalloc(256, 1, 0, _abi.FFT_FLAG_VARIANT(tc), p, p, None) == code["FFT_ERR_INVALID_VALUE"]
    assert L.fft_execute_noalloc(8, 0, 0, 0, None, None, None) == code["FFT_OK"]
    assert L.fft_status_string(code["FFT_ERR_NOALLOC_LIMIT"])
    torch.cuda.synchronize()
