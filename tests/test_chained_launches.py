"""Back-to-back dependent calls on one stream.

Every kernel is launched with programmatic stream serialization (the next
kernel of the stream may be scheduled while the previous one drains) and waits
for its predecessor before it touches memory.  A call that reads the previous
call's output, or overwrites the buffer the previous call reads (in place),
must therefore see that call complete.  Chains of forward and inverse
transforms, on buffers each call hands to the next, must come back to the
input; a missing or misplaced wait shows up as garbage.  The calls move 2^22
elements or more (the programmatic launches) and take a few microseconds each,
so that consecutive launches overlap.
"""
import numpy as np
import pytest
import torch

import synth
from tests.helpers import max_rel_l2

pytestmark = pytest.mark.gpu

import paper_2203_09384_gb300 as gb  # noqa: E402

CHAIN_TOL = 1e-4  # 40 FP32 transforms, each ~1e-7 relative


@pytest.mark.parametrize("n", [8, 32, 64, 128, 256, 512, 1024, 2048])
def test_forward_inverse_chain(n):
    batch = (2 ** 22) // n
    x = synth.uniform(batch, n, seed=31).cuda()
    fwd = gb.Plan(n, batch)
    inv = gb.Plan(n, batch, inverse=True)
    a = x.clone()
    t = torch.empty_like(x)
    for _ in range(10):
        fwd.execute(a, t)  # t = F a
        inv.execute(t, a)  # a = F^-1 t: reads what the previous launch wrote
        fwd.execute(a, a)  # in place: overwrites what it reads
        inv.execute(a, a)
    torch.cuda.synchronize()
    assert fwd.error() == 0 and inv.error() == 0
    err = max_rel_l2(a.cpu().numpy().astype(np.complex128), x.cpu().numpy().astype(np.complex128))
    assert err <= CHAIN_TOL, (n, err)
    fwd.close()
    inv.close()


@pytest.mark.parametrize("dtype", ["tc_f16", "tc_bf16"])
def test_tensor_core_chain(dtype):
    n, batch = 2048, 2048
    x = synth.uniform(batch, n, seed=32).cuda()
    fwd = gb.Plan(n, batch, dtype=dtype)
    inv = gb.Plan(n, batch, inverse=True, dtype=dtype)
    a = x.clone()
    t = torch.empty_like(x)
    for _ in range(3):
        fwd.execute(a, t)
        inv.execute(t, a)
    torch.cuda.synchronize()
    assert fwd.error() == 0 and inv.error() == 0
    err = max_rel_l2(a.cpu().numpy().astype(np.complex128), x.cpu().numpy().astype(np.complex128))
    assert err <= 3e-2, (dtype, err)  # 6 reduced-precision transforms
    fwd.close()
    inv.close()


def test_ragged_chain():
    lengths = synth.ragged_lengths(20000, seed=33)  # 10.1M elements: launched programmatically
    offsets = synth.ragged_offsets(lengths).numpy()
    x = synth.ragged_uniform(lengths, seed=33).cuda()
    fwd = gb.RaggedPlan(offsets)
    inv = gb.RaggedPlan(offsets, inverse=True)
    a = x.clone()
    t = torch.zeros_like(x)
    for _ in range(10):
        fwd.execute(a, t)
        inv.execute(t, a)
        fwd.execute(a, a)
        inv.execute(a, a)
    torch.cuda.synchronize()
    err = max_rel_l2(a.cpu().numpy().astype(np.complex128)[None], x.cpu().numpy().astype(np.complex128)[None])
    assert err <= CHAIN_TOL, err
    fwd.close()
    inv.close()
