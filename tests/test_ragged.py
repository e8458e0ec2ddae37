"""Ragged batches (mixed power-of-two lengths, one persistent launch) and the
autotuner, against the FP64 oracle.

Workload: 20000 signals, lengths 2^u with u uniform on {4..11} (seed 3),
re/im iid U[-1, 1], packed back to back with an offset table.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.helpers import FP32_TOL, max_rel_l2

pytestmark = pytest.mark.gpu

import paper_2203_09384_gb300 as gb  # noqa: E402
from paper_2203_09384_gb300 import _abi, autotune  # noqa: E402


def oracle_ragged(x_flat: np.ndarray, offsets, inverse=False, normalized=True) -> np.ndarray:
    """Per-length batches through the oracle, scattered back into place."""
    offsets = np.asarray(offsets)
    out = np.zeros(x_flat.shape[0], np.complex128)
    lengths = np.diff(offsets)
    for n in np.unique(lengths):
        idx = np.nonzero(lengths == n)[0]
        rows = np.stack([x_flat[offsets[i]:offsets[i] + n] for i in idx]).astype(np.complex128)
        y = oracle.reference(rows, inverse, normalized, threads=8)
        for r, i in enumerate(idx):
            out[offsets[i]:offsets[i] + n] = y[r]
    return out


def per_signal_max_err(got: np.ndarray, want: np.ndarray, offsets) -> float:
    worst = 0.0
    for i in range(len(offsets) - 1):
        a, b = offsets[i], offsets[i + 1]
        worst = max(worst, max_rel_l2(got[None, a:b], want[None, a:b]))
    return worst


@pytest.fixture(scope="module")
def workload():
    lengths = synth.ragged_lengths(20000, seed=3)
    offsets = synth.ragged_offsets(lengths)
    x = synth.ragged_uniform(lengths, seed=3)
    want = oracle_ragged(x.numpy(), offsets.numpy())
    return offsets.numpy(), x, want


@pytest.mark.parametrize("variant", list(range(gb.fft_ragged_variant_count())))
def test_ragged_workload_in_a_cuda_graph(workload, variant):
    offsets, x, want = workload
    xd = x.cuda()
    out = torch.full_like(xd, float("nan"))
    plan = gb.RaggedPlan(offsets, variant=variant)
    info = plan.info()
    assert info.kernel_kind == 3 and info.work_items > 0 and info.batch == len(offsets) - 1
    g = plan.capture(xd, out)
    out.fill_(float("nan"))
    g.replay()
    g.replay()  # replays again: counter variants reset their work counter in a memset node
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.complex128)
    assert per_signal_max_err(got, want, offsets) <= FP32_TOL
    assert _abi.lib().fft_plan_get_error(plan.handle) == 0
    plan.close()


def _per_signal_rel_l2(got: np.ndarray, want: np.ndarray, offsets) -> np.ndarray:
    starts = np.asarray(offsets[:-1])
    num = np.add.reduceat(np.abs(got - want) ** 2, starts)
    den = np.add.reduceat(np.abs(want) ** 2, starts)
    return np.sqrt(num / np.maximum(den, 1e-300))


@pytest.mark.parametrize("variant", list(range(gb.fft_ragged_variant_count())))
def test_many_replays_two_inputs(workload, variant):
    """Two graphs of one plan (different buffers) replayed alternately 24
    times: a race between work items, warp groups or ring slots that a single
    replay does not expose shows up as a wrong result here."""
    offsets, x, want = workload
    xa = x.cuda()
    xb = xa * (0.5 + 0.25j)  # the transform is linear: expected = want * (0.5 + 0.25j)
    oa = torch.full_like(xa, float("nan"))
    ob = torch.full_like(xb, float("nan"))
    plan = gb.RaggedPlan(offsets, variant=variant)
    ga = plan.capture(xa, oa)
    gb_ = plan.capture(xb, ob)
    for _ in range(12):
        ga.replay()
        gb_.replay()
    torch.cuda.synchronize()
    assert _abi.lib().fft_plan_get_error(plan.handle) == 0
    ea = _per_signal_rel_l2(oa.cpu().numpy().astype(np.complex128), want, offsets)
    eb = _per_signal_rel_l2(ob.cpu().numpy().astype(np.complex128), want * (0.5 + 0.25j), offsets)
    assert ea.max() <= FP32_TOL and eb.max() <= FP32_TOL, (variant, ea.max(), eb.max())
    plan.close()


def test_offsets_beyond_2_32_elements():
    """Signals of every length placed on both sides of element 2^32 of one
    34 GB buffer (64-bit offsets), transformed in place by every variant."""
    lengths = np.array([2 ** k for k in range(1, 12)] * 3)
    start = 2 ** 32 - 2 * 2048  # even; the signals straddle element 2^32
    offsets = np.concatenate([[start], start + np.cumsum(lengths)])
    total = int(offsets[-1])
    if torch.cuda.mem_get_info()[0] < 8 * total + (4 << 30):
        pytest.skip("needs about 40 GB of free device memory")
    seg = synth.uniform(1, total - start, seed=23).reshape(-1)
    want = oracle_ragged(seg.numpy(), offsets - start)
    buf = torch.empty(total, dtype=torch.complex64, device="cuda")
    for variant in range(gb.fft_ragged_variant_count()):
        buf[start:].copy_(seg)
        plan = gb.RaggedPlan(offsets, variant=variant)
        plan.execute(buf, buf)
        torch.cuda.synchronize()
        assert _abi.lib().fft_plan_get_error(plan.handle) == 0
        plan.close()
        got = buf[start:].cpu().numpy().astype(np.complex128)
        assert per_signal_max_err(got, want, offsets - start) <= FP32_TOL, variant
    del buf
    torch.cuda.empty_cache()


def test_every_length_mixed_inverse_inplace():
    rng = np.random.default_rng(17)
    lengths = rng.choice([2 ** k for k in range(1, 12)], size=1500)
    lengths = np.concatenate([[2 ** k for k in range(1, 12)], lengths])
    offsets = np.concatenate([[6], 6 + np.cumsum(lengths)])  # even, non-zero start
    x = synth.uniform(1, int(offsets[-1]), seed=18).reshape(-1)
    x[:6] = 0
    for inverse, normalized in [(False, True), (True, True), (True, False)]:
        want = oracle_ragged(x.numpy(), offsets, inverse, normalized)
        for variant in range(gb.fft_ragged_variant_count()):
            xd = x.cuda()
            plan = gb.RaggedPlan(offsets, inverse=inverse, normalized=normalized, variant=variant)
            plan.execute(xd, xd)  # in place
            torch.cuda.synchronize()
            got = xd.cpu().numpy().astype(np.complex128)
            assert per_signal_max_err(got, want, offsets) <= FP32_TOL, (inverse, normalized, variant)
            assert np.all(got[:6] == 0)  # untouched before offsets[0]
            plan.close()


def test_runs_of_equal_lengths():
    """Runs of equal lengths, so that some tiles are one back-to-back span
    (fetched by a single bulk copy, offsets computed) and others are not:
    runs longer and shorter than a tile, broken by other lengths, every
    variant, forward and inverse, against the oracle."""
    rng = np.random.default_rng(41)
    runs = []
    for _ in range(60):
        n = int(2 ** rng.integers(1, 12))
        runs.append(np.full(int(rng.integers(1, 300 if n <= 64 else 12)), n))
    runs.append(np.full(700, 16))  # several whole 16-point tiles
    lengths = np.concatenate(runs)
    offsets = np.concatenate([[2], 2 + np.cumsum(lengths)])
    x = synth.uniform(1, int(offsets[-1]), seed=42).reshape(-1)
    x[:2] = 0
    for inverse in (False, True):
        want = oracle_ragged(x.numpy(), offsets, inverse)
        for variant in range(gb.fft_ragged_variant_count()):
            plan = gb.RaggedPlan(offsets, inverse=inverse, variant=variant)
            y = torch.zeros_like(x).cuda()
            plan.execute(x.cuda(), y)
            torch.cuda.synchronize()
            assert _abi.lib().fft_plan_get_error(plan.handle) == 0
            plan.close()
            got = y.cpu().numpy().astype(np.complex128)
            assert per_signal_max_err(got, want, offsets) <= FP32_TOL, (inverse, variant)
            assert np.all(got[:2] == 0)


def test_ragged_edge_cases():
    # one signal; empty list
    x = synth.uniform(1, 64, seed=1).reshape(-1).cuda()
    p = gb.RaggedPlan([0, 64])
    y = p.execute(x)
    torch.cuda.synchronize()
    assert max_rel_l2(y.cpu().numpy()[None], oracle.reference(x.cpu().numpy()[None])) <= FP32_TOL
    p.close()
    empty = gb.RaggedPlan([0])
    empty.execute(x, torch.empty_like(x))
    empty.close()
    # the library sees bare pointers: a short or misplaced out is refused before launch
    p = gb.RaggedPlan([0, 64])
    with pytest.raises(ValueError):
        p.execute(x, torch.empty(32, dtype=torch.complex64, device="cuda"))
    with pytest.raises(ValueError):
        p.execute(x, torch.empty(64, dtype=torch.complex64))
    with pytest.raises(TypeError):
        p.execute(x, torch.empty(64, dtype=torch.complex128, device="cuda"))
    p.close()
    code = _abi.STATUS_CODE
    for offs, err in [([0, 12], "FFT_ERR_INVALID_SIZE"), ([0, 4096], "FFT_ERR_INVALID_SIZE"),
                      ([0, 1], "FFT_ERR_INVALID_SIZE"), ([1, 9], "FFT_ERR_MISALIGNED"),
                      ([0, 8, 4], "FFT_ERR_INVALID_SIZE")]:
        with pytest.raises(gb.FFTError) as e:
            gb.RaggedPlan(offs)
        assert e.value.status == code[err]
    with pytest.raises(gb.FFTError):
        gb.RaggedPlan([0, 8], variant=gb.fft_ragged_variant_count())


def test_autotuner_picks_a_valid_variant_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("GBFFT_TUNE_CACHE", str(tmp_path / "tune.json"))
    before = {n: gb.fft_get_default_variant(n) for n in (32, 2048)}
    try:
        res = autotune.tune_lengths([32, 2048], elems=2 ** 22, reps=3)
        for n, r in res.items():
            assert 0 <= r["best"] < gb.fft_variant_count(n)
            assert gb.fft_get_default_variant(n) == r["best"]
            assert r["ms"][r["best"]] == min(r["ms"].values())
        lengths = synth.ragged_lengths(500, seed=3)
        offs = synth.ragged_offsets(lengths)
        x = synth.ragged_uniform(lengths, seed=3).cuda()
        rr = autotune.tune_ragged(offs.numpy(), x, torch.empty_like(x), reps=3)
        assert 0 <= rr["best"] < gb.fft_ragged_variant_count()
        path = autotune.save_cache(res, rr)
        for n, v in before.items():
            gb.fft_set_default_variant(n, v)
        entry = autotune.load_cache(path)
        assert entry["plain"] == {str(n): r["best"] for n, r in res.items()}
        assert gb.fft_get_default_variant(2048) == res[2048]["best"]
    finally:
        for n, v in before.items():
            gb.fft_set_default_variant(n, v)
