"""complex32 storage (dtype "c32"): binary16 (re, im) per element with one
power-of-two exponent per signal, FP32 arithmetic inside the kernel.

The oracle transforms the exact values the encoded input holds (stored *
2^exp, in FP64); the kernel's output, decoded the same way, must match it per
signal within the binary16 storage rounding of the output, 2^-11 relative
(round to nearest, 11 significant bits, every component in the normal range
because the exponent puts the largest one in [2^14, 2^15)), plus the FP32
arithmetic tolerance.  Inputs: synth.scaled_normal (N(0,1) signals scaled by
10^u, u ~ U(-3, 3)), batches spanning several blocks and a ragged tail.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.helpers import (FP32_TOL, c32_decode, c32_encode, c32_max_stored, c32_to, every_signal_violations,
                           oracle_max_rel_l2,
                           max_rel_l2, rel_l2_per_signal)

pytestmark = pytest.mark.gpu

import paper_2203_09384_gb300 as gb  # noqa: E402
from paper_2203_09384_gb300 import _abi  # noqa: E402

C32_TOL = 2.0 ** -11 + FP32_TOL
POW2 = [2 ** k for k in range(1, 12)]


def run(xs, xe, n, inverse=False, normalized=True, **kw):
    plan = gb.Plan(n, xs.shape[0], inverse=inverse, normalized=normalized, dtype="c32", **kw)
    try:
        ys, ye = plan.execute_c32(c32_to(xs, "cuda"), xe.cuda())
        torch.cuda.synchronize()
        assert plan.error() == 0
        info = plan.info()
        assert info.dtype == _abi.FFT_C32 and info.kernel_kind == 4
    finally:
        plan.close()
    return c32_to(ys, "cpu"), ye.cpu()


def check_exponents(ys, ye, nonzero):
    m = c32_max_stored(ys)
    assert np.all((m[nonzero] >= 2.0 ** 14) & (m[nonzero] <= 2.0 ** 15)), m[nonzero].min()
    assert np.all(m[~nonzero] == 0) and np.all(ye.numpy()[~nonzero] == 0)


@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("n", POW2)
def test_every_length_against_oracle(n, inverse):
    batch = max(3 * 152 + 7, (1 << 19) // n + 7)
    x, _ = synth.scaled_normal(batch, n, seed=40 + n)
    xs, xe = c32_encode(x.numpy())
    want = oracle.reference(c32_decode(xs, xe), inverse, True, threads=8)
    ys, ye = run(xs, xe, n, inverse)
    err = rel_l2_per_signal(c32_decode(ys, ye), want)
    assert err.max() <= C32_TOL, (n, inverse, err.max())
    assert err.mean() < 4e-4  # typical rounding sits well inside the bound
    check_exponents(ys, ye, np.ones(batch, bool))


def c32_variants(n):
    return [v for v in range(gb.fft_variant_count(n)) if gb.fft_variant_dtype(n, v) == _abi.FFT_C32]


@pytest.mark.parametrize("n,variant", [(n, v) for n in POW2 for v in c32_variants(n)])
def test_every_complex32_schedule(n, variant):
    batch = 2 * 152 * max(1, 4096 // n) + 5
    x, _ = synth.scaled_normal(batch, n, seed=9)
    xs, xe = c32_encode(x.numpy())
    xt = c32_decode(xs, xe)
    for inverse in (False, True):
        ys, ye = run(xs, xe, n, inverse, variant=variant)
        err = rel_l2_per_signal(c32_decode(ys, ye), oracle.reference(xt, inverse, threads=8))
        assert err.max() <= C32_TOL, (n, variant, inverse, err.max())


def test_ring_bounded_wait_reports_timeout():
    n = 2048
    ring = []
    for v in c32_variants(n):
        p = gb.Plan(n, 1, dtype="c32", variant=v)
        if p.info().pipeline > 0:
            ring.append(v)
        p.close()
    assert ring
    batch = 4 * 152 + 3
    xs = torch.zeros(batch, 2 * n, dtype=torch.float16, device="cuda").view(torch.complex32)
    xe = torch.zeros(batch, dtype=torch.int8, device="cuda")
    plan = gb.Plan(n, batch, dtype="c32", variant=ring[0], extra_flags=gb.FFT_FLAG_TEST_STALL)
    plan.set_wait_limit(1_000_000)  # 1 ms
    ys = torch.full((batch, 2 * n), 1.0, dtype=torch.float16, device="cuda").view(torch.complex32)
    ye = torch.full((batch,), 5, dtype=torch.int8, device="cuda")
    plan.execute_c32(xs, xe, ys, ye)
    torch.cuda.synchronize()
    assert plan.error() == _abi.STATUS_CODE["FFT_ERR_TIMEOUT"]
    assert torch.all(ys.view(torch.float16) == 1.0) and torch.all(ye == 5)  # nothing stored
    plan.close()


@pytest.mark.parametrize("n", [2, 64, 2048])
def test_scaling_modes_and_in_place(n):
    batch = 333
    x, _ = synth.scaled_normal(batch, n, seed=7)
    xs, xe = c32_encode(x.numpy())
    xt = c32_decode(xs, xe)
    for inverse, normalized, sf in [(True, False, False), (False, True, True)]:
        ys, ye = run(xs, xe, n, inverse, normalized, scale_forward=sf)
        want = oracle.reference(xt, inverse, normalized, threads=8)
        if sf:
            want = want / n
        assert max_rel_l2(c32_decode(ys, ye), want) <= C32_TOL
    # in place, exponents in place
    plan = gb.Plan(n, batch, dtype="c32")
    d, de = c32_to(xs, "cuda"), xe.cuda()
    plan.execute_c32(d, de, d, de)
    torch.cuda.synchronize()
    plan.close()
    assert max_rel_l2(c32_decode(d, de), oracle.reference(xt, threads=8)) <= C32_TOL


def test_exact_and_degenerate_signals():
    n, batch = 1024, 6
    z = np.zeros((batch, n), np.complex128)
    z[0, 0] = 2.0 ** 17          # delta: flat spectrum 2^17, stored 2^14, exponent 3
    z[1, 0] = -(2.0 ** -100)     # tiny delta: exponent -114
    z[2, 0] = 2.0 ** 100         # huge delta: exponent 86
    z[3, :] = 3.0                # constant: spectrum 3N at bin 0
    # signal 4 stays zero
    z[5] = synth.normal(1, n, seed=3).numpy()[0]
    xs, xe = c32_encode(z)
    xe[4] = 77                   # a zero signal's exponent is free; output exponent 0
    ys, ye = run(xs, xe, n)
    got = c32_decode(ys, ye)
    assert np.array_equal(got[0], np.full(n, 2.0 ** 17))
    assert ye[0] == 3 and ye[1] == -114 and ye[2] == 86
    assert np.array_equal(got[1], np.full(n, -(2.0 ** -100)))
    assert np.array_equal(got[2], np.full(n, 2.0 ** 100))
    assert got[3, 0] == 3.0 * n and np.all(got[3, 1:] == 0)
    assert np.all(got[4] == 0) and ye[4] == 0
    assert max_rel_l2(got[5:], oracle.reference(z[5:])) <= C32_TOL
    check_exponents(ys, ye, np.array([1, 1, 1, 1, 0, 1], bool))


@pytest.mark.parametrize("n", [256, 2048])
def test_full_size_every_signal(n):
    """The benchmark's complex32 workload: N * batch = 2^28 elements (1 GiB in),
    U[-1, 1] (seed n) encoded to complex32.  Input and output are decoded on
    the device to complex64 (exact for these exponents) and EVERY signal is
    compared element by element with the FP64 oracle's transform of the
    values the input encoding holds; every signal also against Parseval and
    the bins 0 and N/2."""
    batch = 2 ** 28 // n
    x = synth.uniform(batch, n, seed=n, device="cuda")
    xs, xe = c32_encode_device(x)
    del x
    plan = gb.Plan(n, batch, dtype="c32")
    ys, ye = plan.execute_c32(xs, xe)
    torch.cuda.synchronize()
    assert plan.error() == 0
    plan.close()
    xd, yd = c32_decode_c64(xs, xe), c32_decode_c64(ys, ye)
    del xs, ys
    err, where = oracle_max_rel_l2(xd, yd)
    assert err <= C32_TOL, (n, err, where)
    bad = every_signal_violations(xd, yd, C32_TOL)
    assert bad.numel() == 0, bad[:8]
    del xd, yd
    torch.cuda.empty_cache()


def c32_decode_c64(stored: torch.Tensor, exp: torch.Tensor) -> torch.Tensor:
    """complex32 storage decoded on the device to complex64: exact while the
    exponents keep every value inside FP32's normal range."""
    assert int(exp.abs().max()) < 100
    h = stored.view(torch.float16).reshape(stored.shape[0], -1, 2).float()
    h = h * torch.pow(2.0, exp.float())[:, None, None]
    return torch.view_as_complex(h)


def c32_encode_device(x: torch.Tensor):
    """c32_encode on the device in torch ops (same exponent rule), for inputs
    too large to move through numpy."""
    ri = torch.view_as_real(x)
    m = ri.abs().amax(dim=(1, 2)).double()
    e = torch.where(m > 0, torch.frexp(m)[1] - 15, torch.zeros_like(m, dtype=torch.int32))
    h = (ri.double() * torch.pow(2.0, -e.double())[:, None, None]).half()
    return h.reshape(x.shape[0], -1).view(torch.complex32), e.to(torch.int8)


def test_rejections():
    code = _abi.STATUS_CODE
    x = torch.zeros(64, 8, dtype=torch.float16, device="cuda").view(torch.complex32)
    e = torch.zeros(64, dtype=torch.int8, device="cuda")
    c32 = gb.Plan(4, 64, dtype="c32")
    c64 = gb.Plan(4, 64)
    L = _abi.lib()
    s = torch.cuda.current_stream().cuda_stream
    assert L.fft_execute(c32.handle, x.data_ptr(), x.data_ptr(), s) == code["FFT_ERR_INVALID_VALUE"]
    assert L.fft_execute_c32(c64.handle, x.data_ptr(), e.data_ptr(), x.data_ptr(), e.data_ptr(), s) == \
        code["FFT_ERR_INVALID_VALUE"]
    assert L.fft_execute_c32(c32.handle, x.data_ptr() + 4, e.data_ptr(), x.data_ptr() + 4, e.data_ptr(), s) == \
        code["FFT_ERR_MISALIGNED"]
    assert L.fft_execute_c32(c32.handle, x.data_ptr(), e.data_ptr(), x.data_ptr() + 16, e.data_ptr(), s) == \
        code["FFT_ERR_OVERLAP"]
    assert L.fft_execute_c32(c32.handle, x.data_ptr(), e.data_ptr(), x.data_ptr(), e.data_ptr() + 1, s) == \
        code["FFT_ERR_OVERLAP"]
    assert L.fft_execute_c32(c32.handle, x.data_ptr(), None, x.data_ptr(), e.data_ptr(), s) == \
        code["FFT_ERR_INVALID_VALUE"]
    with pytest.raises(gb.FFTError):
        c32.execute(torch.zeros(64, 4, dtype=torch.complex64, device="cuda"))
    c32.close()
    c64.close()
    with pytest.raises(gb.FFTError) as err:
        _abi.fft_plan_create_ex(64, 8, 0, _abi.FFT_C32, _abi.FFT_FLAG_HOST_STAGING)
    assert err.value.name == "FFT_ERR_UNSUPPORTED"
    v32 = c32_variants(64)
    assert len(v32) >= 1
    with pytest.raises(gb.FFTError):
        gb.Plan(64, 8, variant=v32[0])  # complex64 plan on the complex32 kernel
    with pytest.raises(gb.FFTError):
        gb.Plan(64, 8, variant=0, dtype="c32")  # complex32 plan on a complex64 kernel
    with pytest.raises(gb.FFTError):
        gb.fft_set_default_variant(64, v32[0])
    torch.cuda.synchronize()
