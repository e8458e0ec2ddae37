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


def test_plan_cache_is_a_bounded_lru(monkeypatch):
    """get_plan keeps at most PLAN_CACHE_SIZE plans: the least recently used
    one is retired (its device synchronised, then the plan closed) when a new
    shape comes in; a hit moves a plan to the most recent end."""
    made, retired = [], []

    class FakePlan:
        def __init__(self, n, batch, *a, **k):
            self.key = (n, batch)
            made.append(self.key)

        def close(self):
            retired.append(self.key)

    monkeypatch.setattr(gb, "Plan", FakePlan)
    monkeypatch.setattr(gb, "_retire", lambda p: p.close())
    monkeypatch.setattr(gb, "PLAN_CACHE_SIZE", 3)
    monkeypatch.setattr(gb, "_cache", gb.collections.OrderedDict())
    get = lambda b: gb.get_plan(64, b, False, True, "cuda:0")  # noqa: E731
    a = get(1)
    get(2)
    get(3)
    assert get(1) is a and made == [(64, 1), (64, 2), (64, 3)]  # a hit makes no plan
    get(4)  # evicts batch 2, the least recently used
    assert retired == [(64, 2)] and len(gb._cache) == 3
    get(5)
    assert retired == [(64, 2), (64, 3)]
    assert get(1) is a
    gb.clear_plan_cache()
    assert sorted(retired) == sorted([(64, 1), (64, 2), (64, 3), (64, 4), (64, 5)]) and not gb._cache
