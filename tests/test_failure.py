"""Failure detection without a GPU fault: bounded device-side waits.

The test-only plan flag FFT_FLAG_TEST_STALL makes the kernels that wait on the
device (the bulk-copy prefetch ring, the tensor-core MMA completion) issue
nothing, so each wait runs out after the plan's wait limit (1 ms here), the
kernel records FFT_ERR_TIMEOUT in the plan's error word and finishes.  The
context must stay usable afterwards.
"""
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
# variant 13 the one with one separate exchange buffer.
@pytest.mark.parametrize("n,dtype,variant", [(2048, "c64", None), (1024, "c64", None), (256, "tc_f16", None),
                                             (2048, "tc_bf16", None), (2048, "c64", 10), (1024, "tc_f16", 11),
                                             (2048, "tc_f16", 13)])
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


def test_kernels_without_waits_ignore_the_test_flag():
    x = synth.uniform(100, 64, seed=2).cuda()
    plan = gb.Plan(64, 100, extra_flags=gb.FFT_FLAG_TEST_STALL)
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
