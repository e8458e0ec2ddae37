"""The GBFFT_DEBUG build of the library (``build(debug=True)``, its own
``_build_debug/libgbfft.so``), which the package never loads: every
shared-memory exchange index, stage-0 tile read, global element index and
twiddle index is checked on the device, a failed check records
FFT_ERR_DEVICE_CHECK in the plan's error word instead of faulting, and every
exchange slot is poisoned with NaN once read, so a slot a later stage fails to
write reaches the output.  Every compiled schedule (FP32, tensor-core,
complex32), every ragged variant and the allocation-free entry point run
through it here: no check may fire and every result must match the FP64
oracle.  This stands in for a memory checker, which is not available here.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.helpers import FP32_TOL, c32_decode, c32_encode, c32_to, max_rel_l2, to_np

pytestmark = pytest.mark.gpu

from paper_2203_09384_gb300 import _abi  # noqa: E402
from paper_2203_09384_gb300 import build as gbuild  # noqa: E402

OK = 0
TC_TOL = 5e-3
C32_TOL = 2.0 ** -11 + 1e-5


@pytest.fixture(scope="module")
def dlib():
    path = gbuild.build(debug=True)
    assert path != _abi.LIB_PATH
    return _abi.declare(ctypes.CDLL(path))


def _rows():
    out = []
    for k in range(1, 12):
        n = 2 ** k
        for v in range(_abi.fft_variant_count(n)):
            out.append((n, v, _abi.fft_variant_dtype(n, v)))
    return out


def _plan(L, n, batch, direction, dtype, flags):
    h = ctypes.c_void_p()
    assert L.fft_plan_create_ex(n, batch, direction, dtype, flags, ctypes.byref(h)) == OK
    return h


@pytest.mark.parametrize("n,variant,dtype", _rows())
def test_every_schedule_passes_the_device_checks(dlib, n, variant, dtype):
    batch = 4096 + 3  # every ring wraps, and the last tile is ragged
    flags = _abi.FFT_FLAG_VARIANT(variant)
    s = torch.cuda.current_stream().cuda_stream
    for direction in (_abi.FFT_FORWARD, _abi.FFT_INVERSE):
        inverse = direction == _abi.FFT_INVERSE
        h = _plan(dlib, n, batch, direction, dtype, flags)
        try:
            if dtype == _abi.FFT_C32:
                x = synth.uniform(batch, n, seed=60 + variant)
                xs, xe = c32_encode(x)
                xsd, xed = c32_to(xs, "cuda"), xe.cuda()
                ys = torch.empty_like(xsd)
                ye = torch.empty_like(xed)
                assert dlib.fft_execute_c32(h, xsd.data_ptr(), xed.data_ptr(), ys.data_ptr(), ye.data_ptr(), s) == OK
                torch.cuda.synchronize()
                got, src, tol = c32_decode(ys, ye), c32_decode(xs, xe), C32_TOL
            else:
                if dtype == _abi.FFT_C64:
                    x, tol = synth.uniform(batch, n, seed=60 + variant), FP32_TOL
                else:
                    x, _ = synth.scaled_normal(batch, n, seed=60 + variant)
                    tol = TC_TOL
                xd = x.cuda()
                y = torch.empty_like(xd)
                assert dlib.fft_execute(h, xd.data_ptr(), y.data_ptr(), s) == OK
                torch.cuda.synchronize()
                got, src = to_np(y), x.numpy()
            assert dlib.fft_plan_get_error(h) == OK, (n, variant, direction)
        finally:
            dlib.fft_plan_destroy(h)
        assert not np.isnan(got).any(), (n, variant, direction)
        assert max_rel_l2(got, oracle.reference(src, inverse, threads=8)) <= tol, (n, variant, direction)


@pytest.mark.parametrize("variant", list(range(_abi.fft_ragged_variant_count())))
def test_every_ragged_variant_passes_the_device_checks(dlib, variant):
    rng = np.random.default_rng(71)
    lengths = rng.choice([2 ** k for k in range(1, 12)], size=3000)
    offsets = np.concatenate([[6], 6 + np.cumsum(lengths)]).astype(np.int64)
    x = synth.uniform(1, int(offsets[-1]), seed=72).reshape(-1)
    xd = x.cuda()
    y = torch.full_like(xd, float("nan"))
    arr = (ctypes.c_int64 * len(offsets))(*offsets.tolist())
    h = ctypes.c_void_p()
    assert dlib.fft_plan_create_ragged(arr, len(offsets) - 1, 0, 0, _abi.FFT_FLAG_VARIANT(variant),
                                       ctypes.byref(h)) == OK
    try:
        assert dlib.fft_execute(h, xd.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream) == OK
        torch.cuda.synchronize()
        assert dlib.fft_plan_get_error(h) == OK
    finally:
        dlib.fft_plan_destroy(h)
    got = to_np(y)
    for n in np.unique(lengths):
        idx = np.nonzero(lengths == n)[0]
        rows = np.stack([x.numpy()[offsets[i]:offsets[i] + n] for i in idx])
        want = oracle.reference(rows, threads=8)
        have = np.stack([got[offsets[i]:offsets[i] + n] for i in idx])
        assert max_rel_l2(have, want) <= FP32_TOL, (variant, n)


def test_allocation_free_entry_point_passes_the_device_checks(dlib):
    """fft_execute_noalloc of the debug build: its kernels' checks record into
    the static array's error word, which the next call clears, so here the
    check is that the results are right and free of poison."""
    s = torch.cuda.current_stream().cuda_stream
    for n, batch in ((2048, 1001), (256, 3003), (8, 5005)):
        x = synth.uniform(batch, n, seed=n).cuda()
        y = torch.empty_like(x)
        assert dlib.fft_execute_noalloc(n, batch, 0, 0, x.data_ptr(), y.data_ptr(), s) == OK
        torch.cuda.synchronize()
        got = to_np(y)
        assert not np.isnan(got).any()
        assert max_rel_l2(got, oracle.reference(x.cpu().numpy(), threads=8)) <= FP32_TOL
