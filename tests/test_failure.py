"""Failure detection without a GPU fault: bounded device-side waits.

The test-only plan flag FFT_FLAG_TEST_STALL makes the kernels that wait on the
device (the bulk-copy prefetch rings, ragged variants 4 and up, the tensor-core MMA
completion) issue nothing, so each wait runs out after the plan's wait limit (1 ms here), the
kernel records FFT_ERR_TIMEOUT in the plan's error word and finishes.  The
context must stay usable afterwards.
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

TIMEOUT = _abi.STATUS_CODE["FFT_ERR_TIMEOUT"]


# (n, dtype, schedule variant or None for the default).  At N = 2048 the
# default FP32 schedule, at N = 1024 / 2048 the default tensor-core schedules
# and variant 11 (FP16) are ring kernels that exchange inside the ring slot;
# variant 10 of N = 2048 is the ring kernel with two exchange buffers and
# variant 13 the one with one separate exchange buffer; the N = 64 and 128
# defaults place their signals apart in the ring slot (copies by warp 0).
@pytest.mark.parametrize("n,dtype,variant", [(2048, "c64", None), (1024, "c64", None), (256, "tc_f16", None),
                                             (2048, "tc_bf16", None), (2048, "c64", 10), (1024, "tc_f16", 11),
                                             (2048, "tc_f16", 13), (64, "c64", None), (128, "c64", None)])
def test_bounded_wait_reports_timeout(n, dtype, variant):
    batch = 4 * 152 + 3
    x = synth.uniform(batch, n, seed=1).cuda()
    out = torch.zeros_like(x)
    plan = gb.Plan(n, batch, dtype=dtype, variant=variant, extra_flags=gb.FFT_FLAG_TEST_STALL)
    info = plan.info()
    assert info.kernel_kind == 2 or info.tc != 0  # a kernel with device-side waits
    plan.set_wait_limit(1_000_000)  # 1 ms
    plan.execute(x, out)
    torch.cuda.synchronize()
    assert plan.error() == TIMEOUT
    assert plan.error() == 0  # reading clears the word
    assert torch.count_nonzero(out) == 0  # nothing was stored
    plan.close()
    # the context is still good: a normal plan gives the right answer
    good = gb.Plan(n, batch, dtype=dtype, variant=variant)
    y = good.execute(x)
    torch.cuda.synchronize()
    assert good.error() == 0
    tol = FP32_TOL if dtype == "c64" else 5e-3
    assert max_rel_l2(to_np(y[:64]), oracle.reference(x[:64].cpu().numpy())) <= tol
    good.close()


def test_error_word_is_read_after_work_on_a_non_blocking_stream():
    """fft_plan_get_error synchronises the plan's device, so a stalled kernel
    enqueued on a non-blocking side stream has finished (and recorded its
    timeout) before the word is read; the caller does no sync of its own."""
    n, batch = 2048, 2 * 152 + 1
    x = synth.uniform(batch, n, seed=3).cuda()
    out = torch.zeros_like(x)
    plan = gb.Plan(n, batch, extra_flags=gb.FFT_FLAG_TEST_STALL)
    plan.set_wait_limit(50_000_000)  # 50 ms: still running when the host asks
    side = torch.cuda.Stream()  # created cudaStreamNonBlocking
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.execute(x, out, stream=side)
    assert plan.error() == TIMEOUT
    assert plan.error() == 0
    assert torch.count_nonzero(out) == 0
    plan.close()


def _ragged_offsets():
    lengths = synth.ragged_lengths(3000, seed=13)
    return synth.ragged_offsets(lengths).numpy()


@pytest.mark.parametrize("variant", list(range(4, gb.fft_ragged_variant_count())))
def test_ragged_bounded_wait_reports_timeout(variant):
    """The ragged variants that wait on the device (the bulk-copy ring, the
    producer warp's ring slots): under the test flag nothing is copied, each
    block's first wait runs out after the plan's 1 ms limit, the word reads
    FFT_ERR_TIMEOUT once, nothing is stored, and the context stays usable."""
    offsets = _ragged_offsets()
    total = int(offsets[-1])
    x = synth.uniform(1, total, seed=5).reshape(-1).cuda()
    out = torch.zeros_like(x)
    plan = gb.RaggedPlan(offsets, variant=variant, extra_flags=gb.FFT_FLAG_TEST_STALL)
    plan.set_wait_limit(1_000_000)
    plan.execute(x, out)
    assert plan.error() == TIMEOUT
    assert plan.error() == 0
    assert torch.count_nonzero(out) == 0
    plan.close()
    good = gb.RaggedPlan(offsets, variant=variant)
    y = good.execute(x)
    assert good.error() == 0
    first = slice(int(offsets[0]), int(offsets[1]))
    want = oracle.reference(x[first].cpu().numpy()[None])
    assert max_rel_l2(to_np(y[first])[None], want) <= FP32_TOL
    good.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_ragged_variants_without_waits_ignore_the_test_flag(variant):
    offsets = _ragged_offsets()[:201]
    x = synth.uniform(1, int(offsets[-1]), seed=6).reshape(-1).cuda()
    plan = gb.RaggedPlan(offsets, variant=variant, extra_flags=gb.FFT_FLAG_TEST_STALL)
    plan.set_wait_limit(1_000_000)
    y = plan.execute(x)
    assert plan.error() == 0
    first = slice(int(offsets[0]), int(offsets[1]))
    assert max_rel_l2(to_np(y[first])[None], oracle.reference(x[first].cpu().numpy()[None])) <= FP32_TOL
    plan.close()


def test_kernels_without_waits_ignore_the_test_flag():
    x = synth.uniform(100, 512, seed=2).cuda()
    plan = gb.Plan(512, 100, extra_flags=gb.FFT_FLAG_TEST_STALL)  # the direct kernel: no device waits
    assert plan.info().pipeline == 0
    y = plan.execute(x)
    torch.cuda.synchronize()
    assert plan.error() == 0
    assert max_rel_l2(to_np(y), oracle.reference(x.cpu().numpy())) <= FP32_TOL
    plan.close()


def test_wait_limit_validation():
    plan = gb.Plan(2048, 8)
    with pytest.raises(gb.FFTError):
        plan.set_wait_limit(0)
    plan.close()


@pytest.mark.parametrize("kind,k", [("plain", 1), ("staging", 1), ("staging", 2), ("ragged", 1)])
def test_every_allocation_failure_of_plan_creation(kind, k, monkeypatch):
    """GBFFT_TEST_FAIL_ALLOC=k (a host-side test hook) makes the k-th device
    allocation of a plan-creation call fail without allocating.  Each failure
    path returns FFT_ERR_ALLOC, frees what the call had already allocated (200
    failing calls leave the device's free memory where it was), and the next
    plan, made without the hook, is correct."""
    n, batch = 256, 4096
    offsets = np.concatenate([[0], np.cumsum([256, 2048, 16] * 10)])

    def create():
        if kind == "ragged":
            return gb.RaggedPlan(offsets)
        return gb.Plan(n, batch, host_staging=kind == "staging")

    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("GBFFT_TEST_FAIL_ALLOC", str(k))
    for _ in range(200):
        with pytest.raises(gb.FFTError) as e:
            create()
        assert e.value.status == _abi.STATUS_CODE["FFT_ERR_ALLOC"]
    monkeypatch.setenv("GBFFT_TEST_FAIL_ALLOC", str(k + 2))  # past the call's last allocation: no failure
    create().close()
    monkeypatch.delenv("GBFFT_TEST_FAIL_ALLOC")
    torch.cuda.synchronize()
    assert free_before - torch.cuda.mem_get_info()[0] < (4 << 20)
    plan = create()
    if kind == "ragged":
        x = synth.uniform(1, int(offsets[-1]), seed=9).reshape(-1).cuda()
        y = plan.execute(x)
        first = slice(0, 256)
        assert max_rel_l2(to_np(y[first])[None], oracle.reference(x[first].cpu().numpy()[None])) <= FP32_TOL
    else:
        x = synth.uniform(batch, n, seed=9).cuda()
        y = plan.execute(x)
        assert max_rel_l2(to_np(y[:32]), oracle.reference(x[:32].cpu().numpy())) <= FP32_TOL
    assert plan.error() == 0
    plan.close()
