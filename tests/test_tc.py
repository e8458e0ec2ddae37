"""FP16 / BF16 tensor-core radix-16 stages (tcgen05) against the FP64 oracle.

Workload: complex N(0,1) signals, each scaled by 10^u with u ~ U(-3, 3)
(seed 4), so that a fixed FP16 range would overflow or underflow without the
power-of-two prescale of the FP16 path (BF16 shares FP32's exponent range).
Bar: per-signal relative L2 <= 5e-3.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.helpers import every_signal_violations, max_rel_l2, oracle_max_rel_l2, rel_l2_per_signal, to_np

pytestmark = pytest.mark.gpu

import paper_2203_09384_gb300 as gb  # noqa: E402

TC_TOL = 5e-3
TC_LENGTHS = [128, 256, 1024, 2048]


def run(x, n, dtype, inverse=False):
    plan = gb.Plan(n, x.shape[0], inverse=inverse, dtype=dtype)
    out = plan.execute(x)
    torch.cuda.synchronize()
    assert plan.error() == 0
    info = plan.info()
    plan.close()
    return out, info


@pytest.mark.parametrize("dtype", ["tc_f16", "tc_bf16"])
@pytest.mark.parametrize("n", TC_LENGTHS)
@pytest.mark.parametrize("inverse", [False, True])
def test_tc_against_oracle(n, dtype, inverse):
    batch = 3 * 152 + 7
    x, _ = synth.scaled_normal(batch, n, seed=4)
    out, info = run(x.cuda(), n, dtype, inverse)
    assert info.tc == (1 if dtype == "tc_f16" else 2)
    err = rel_l2_per_signal(to_np(out), oracle.reference(x.numpy(), inverse, threads=8))
    assert err.max() <= TC_TOL, (n, dtype, err.max())


@pytest.mark.parametrize("dtype", ["tc_f16", "tc_bf16"])
@pytest.mark.parametrize("n", [256, 2048])
def test_precision_workload_every_signal(n, dtype):
    """N in {256, 2048}, batch 2^17, as the benchmark runs it: EVERY signal of
    the batch against the FP64 oracle, element by element (a chunk of 2^24
    elements at a time); every signal also against Parseval and the bins 0
    and N/2 as a cheap extra."""
    batch = 2 ** 17
    x, _ = synth.scaled_normal(batch, n, seed=4, device="cuda")
    out, _ = run(x, n, dtype)
    err, where = oracle_max_rel_l2(x, out)
    assert err <= TC_TOL, (n, dtype, err, where)
    bad = every_signal_violations(x, out, TC_TOL)
    assert bad.numel() == 0, bad[:8]
    del x, out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["tc_f16", "tc_bf16"])
def test_tc_exact_cases(dtype):
    """Inputs whose products are exact in FP16/BF16: delta -> all ones; the
    FP16 prescale is a power of two and BF16 shares FP32's range, so huge and
    tiny deltas come out exact too."""
    for n in TC_LENGTHS:
        for amp in (1.0, 2.0 ** 40, 2.0 ** -40):
            d = synth.delta(n, 0, batch=3) * amp
            out, _ = run(d.cuda(), n, dtype)
            assert torch.equal(out.cpu(), torch.full((3, n), amp, dtype=torch.complex64))
        z = torch.zeros(2, n, dtype=torch.complex64)
        out, _ = run(z.cuda(), n, dtype)
        assert torch.count_nonzero(out) == 0


def test_lengths_without_radix16_stage_run_fp32():
    x = synth.uniform(40, 64, seed=2)
    out, info = run(x.cuda(), 64, "tc_f16")
    assert info.tc == 0
    assert max_rel_l2(to_np(out), oracle.reference(x.numpy())) <= 1e-5


def test_tc_accuracy_is_reported_not_hidden():
    """FP16 must beat BF16 by a wide margin on the same data (2^-11 vs 2^-8
    operand rounding); both stay under the 5e-3 bar."""
    x, _ = synth.scaled_normal(512, 256, seed=4)
    want = oracle.reference(x.numpy(), threads=8)
    e16 = max_rel_l2(to_np(run(x.cuda(), 256, "tc_f16")[0]), want)
    e_bf = max_rel_l2(to_np(run(x.cuda(), 256, "tc_bf16")[0]), want)
    e32 = max_rel_l2(to_np(run(x.cuda(), 256, "c64")[0]), want)
    assert e32 < 1e-6 < e16 < e_bf <= TC_TOL, (e32, e16, e_bf)


def _tc_variants():
    out = []
    for n in [2 ** k for k in range(1, 12)]:
        for v in range(gb.fft_variant_count(n)):
            dt = gb.fft_variant_dtype(n, v)
            if dt in (gb.FFT_C64_TC_F16, gb.FFT_C64_TC_BF16):
                out.append((n, v, gb.DTYPE_NAMES[dt]))
    return out


def _expected_tc_stages(n, variant):
    """From the schedule table: TC & 4 puts only the last radix-16 stage on
    the tensor cores, else every radix-16 stage."""
    from tests.test_bank_model import _rows
    for L, v, E, S, r0, r1, r2, r3, minb, pipe, tc, xb, ch in _rows("GBFFT_GENERIC_SCHEDULES", 13):
        if 2 ** L == n and v == variant:
            sixteen = [r for r in (r0, r1, r2, r3) if r == 16]
            return (1 if sixteen else 0) if tc & 4 else len(sixteen)
    raise KeyError((n, variant))


@pytest.mark.parametrize("n,variant,dtype", _tc_variants())
def test_every_tensor_core_schedule(n, variant, dtype):
    batch = 2 * 152 + 5
    x, _ = synth.scaled_normal(batch, n, seed=6)
    for inverse in (False, True):
        plan = gb.Plan(n, batch, inverse=inverse, dtype=dtype, variant=variant)
        out = plan.execute(x.cuda())
        torch.cuda.synchronize()
        assert plan.error() == 0 and plan.info().variant == variant
        assert plan.info().tc_stages == _expected_tc_stages(n, variant)
        plan.close()
        err = rel_l2_per_signal(to_np(out), oracle.reference(x.numpy(), inverse, threads=8))
        assert err.max() <= TC_TOL, (n, variant, dtype, inverse, err.max())
