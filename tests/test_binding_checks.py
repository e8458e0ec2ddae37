"""Python binding: buffers go to the C-ABI as bare pointers, so their dtype,
layout, device and size are checked before any launch (CPU only)."""
import pytest
import torch

import paper_2203_09384_gb300 as gb

cpu = torch.device("cpu")


def test_check_buffer_accepts_a_matching_buffer():
    gb._check_buffer(torch.zeros(12, dtype=torch.complex64), "x", torch.complex64, cpu, 12)
    gb._check_buffer(torch.zeros(20, dtype=torch.complex64), "x", torch.complex64, cpu, 12, at_least=True)


def test_check_buffer_refuses_mismatches():
    good = torch.zeros(4, 3, dtype=torch.complex64)
    with pytest.raises(TypeError):
        gb._check_buffer(good.to(torch.complex128), "x", torch.complex64, cpu, 12)
    with pytest.raises(ValueError, match="contiguous"):
        gb._check_buffer(good.t(), "x", torch.complex64, cpu, 12)
    with pytest.raises(ValueError, match="elements"):
        gb._check_buffer(good, "out", torch.complex64, cpu, 16)
    with pytest.raises(ValueError, match="at least"):
        gb._check_buffer(good, "out", torch.complex64, cpu, 16, at_least=True)
    with pytest.raises(ValueError, match="expected"):
        gb._check_buffer(torch.zeros(12, dtype=torch.complex64, device="meta"), "x", torch.complex64, cpu, 12)


def test_plans_need_a_cuda_device():
    with pytest.raises(ValueError):
        gb._cuda_device("cpu")
    assert gb._cuda_device("cuda:3") == torch.device("cuda", 3)
