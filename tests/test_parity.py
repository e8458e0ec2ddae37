"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Inputs come from ``synth`` (seeded); expected values from ``oracle`` only.
Pass bar: per-signal relative L2 <= 1e-5 (FP32), max over signals.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.helpers import FP32_TOL, every_signal_violations, max_rel_l2, oracle_max_rel_l2, to_np
from tests.oracle_pins import ramp_closed_form

pytestmark = pytest.mark.gpu

import paper_2203_09384_gb300 as gb  # noqa: E402
from paper_2203_09384_gb300 import _abi  # noqa: E402

POW2 = [2 ** k for k in range(1, 12)]


def run(x_cpu: torch.Tensor, inverse=False, normalized=True, inplace=False, scale_forward=False,
        variant=None):
    """Copy to the GPU, run one planned transform through the C-ABI, copy back."""
    batch, n = x_cpu.shape
    d = x_cpu.to("cuda")
    plan = gb.Plan(n, batch, inverse=inverse, normalized=normalized, scale_forward=scale_forward,
                   variant=variant)
    out = d if inplace else torch.empty_like(d)
    plan.execute(d, out)
    torch.cuda.synchronize()
    assert plan.error() == 0
    res = out.cpu()
    plan.close()
    return res


def oracle_of(x_cpu, inverse=False, normalized=True):
    return oracle.reference(x_cpu.numpy().astype(np.complex128), inverse, normalized, threads=8)


def test_config1_forward_inverse_round_trip():
    """N = 64, batch = 16, re/im iid U[-1, 1], seed 0."""
    x = synth.uniform(16, 64, seed=0)
    X = run(x)
    assert max_rel_l2(to_np(X), oracle_of(x)) <= FP32_TOL
    xi = run(x, inverse=True)
    assert max_rel_l2(to_np(xi), oracle_of(x, inverse=True)) <= FP32_TOL
    back = run(X, inverse=True)
    assert max_rel_l2(to_np(back), x.numpy()) <= FP32_TOL


def _batch_for(n):
    # several blocks of every kernel shape plus a ragged tail
    return max(4, min(1500, 2 ** 19 // (n * n) + 700)) + 3


def _variants():
    return [(n, v) for n in POW2 for v in range(gb.fft_variant_count(n))
            if gb.fft_variant_dtype(n, v) == gb.FFT_C64]


@pytest.mark.parametrize("n,variant", _variants())
@pytest.mark.parametrize("inverse", [False, True])
def test_every_length_and_schedule(n, variant, inverse):
    batch = _batch_for(n)
    x = synth.uniform(batch, n, seed=100 + n)
    want = oracle_of(x, inverse)
    y = run(x, inverse=inverse, variant=variant)
    err = max_rel_l2(to_np(y), want)
    assert err <= FP32_TOL, err
    # accuracy alarm: with exact twiddles FP32 error stays near 1e-7
    assert err <= 1e-6, err
    # a batch too small to fill one block, and one that leaves a ragged tail
    for b in (1, 3 * 152 + 5):
        xs = synth.uniform(b, n, seed=200 + n)
        ys = run(xs, inverse=inverse, variant=variant)
        assert max_rel_l2(to_np(ys), oracle_of(xs, inverse)) <= FP32_TOL


def _ring_candidates():
    """Every non-complex32 schedule of the lengths that have bulk-copy-ring
    schedules (whether a schedule uses the ring is known only from a plan)."""
    out = []
    for n in (128, 256, 1024, 2048):
        for v in range(gb.fft_variant_count(n)):
            dt = gb.fft_variant_dtype(n, v)
            if dt != gb.FFT_C32:
                out.append((n, v, gb.DTYPE_NAMES[dt]))
    return out


@pytest.mark.parametrize("n,variant,dtype", _ring_candidates())
def test_ring_schedules_wrap_their_ring(n, variant, dtype):
    """Every block of a bulk-copy-ring schedule goes round its ring of D slots
    more than twice (slot reuse, refills, mbarrier phase flips) and the batch
    ends on a ragged tile; the last tiles, first signals and a seeded sample
    are checked against the oracle."""
    probe = gb.Plan(n, 2 ** 22 // n, dtype=dtype, variant=variant)
    info = probe.info()
    probe.close()
    if info.pipeline == 0:
        pytest.skip("schedule without a bulk-copy ring")
    resident, s = info.grid, info.signals_per_block  # the grid is capped at the resident blocks
    batch = resident * s * (2 * info.pipeline + 1) + s // 2 + 1
    if dtype == "c64":
        x = synth.uniform(batch, n, seed=300 + variant, device="cuda")
        tol = FP32_TOL
    else:
        x, _ = synth.scaled_normal(batch, n, seed=300 + variant)
        x = x.cuda()
        tol = 5e-3
    for inverse in (False, True):
        plan = gb.Plan(n, batch, inverse=inverse, dtype=dtype, variant=variant)
        assert plan.info().grid == resident
        out = plan.execute(x)
        torch.cuda.synchronize()
        assert plan.error() == 0
        plan.close()
        rng = np.random.default_rng(variant)
        idx = np.unique(np.concatenate([np.arange(4), np.arange(batch - 2 * s - 64, batch),
                                        rng.integers(0, batch, 256)]))
        ti = torch.from_numpy(idx).cuda()
        xs = x.index_select(0, ti).cpu()
        got = to_np(out.index_select(0, ti))
        assert max_rel_l2(got, oracle_of(xs, inverse)) <= tol, (n, variant, dtype, inverse)


@pytest.mark.parametrize("n", [2 ** k for k in range(3, 12)])
def test_paper_ramp(n):
    """The paper's input f(x) = x (Sec. 6) against its closed-form DFT."""
    x = synth.ramp(n, batch=3)
    y = to_np(run(x))
    want = np.broadcast_to(ramp_closed_form(n), y.shape)
    assert max_rel_l2(y, want) <= FP32_TOL
    assert max_rel_l2(y, oracle_of(x)) <= FP32_TOL
    yi = to_np(run(x, inverse=True))
    assert max_rel_l2(yi, np.broadcast_to(ramp_closed_form(n, inverse=True), yi.shape)) <= FP32_TOL


@pytest.mark.parametrize("n", POW2)
def test_round_trip_and_unnormalized(n):
    x = synth.uniform(37, n, seed=7)
    X = run(x)
    back = run(X, inverse=True)
    assert max_rel_l2(to_np(back), x.numpy()) <= FP32_TOL
    adj = run(X, inverse=True, normalized=False)
    assert max_rel_l2(to_np(adj), n * x.numpy().astype(np.complex128)) <= FP32_TOL
    fs = run(x, scale_forward=True)
    assert max_rel_l2(to_np(fs), oracle_of(x) / n) <= FP32_TOL


@pytest.mark.parametrize("n", POW2)
def test_special_inputs(n):
    zero = torch.zeros(5, n, dtype=torch.complex64)
    assert torch.count_nonzero(run(zero)) == 0
    d = synth.delta(n, 0, batch=2)
    assert torch.allclose(run(d), torch.ones(2, n, dtype=torch.complex64), atol=0, rtol=0)
    k = torch.arange(n, dtype=torch.float64)
    m = max(1, n // 3)
    tone = torch.exp(2j * torch.pi * ((k * m) % n) / n).to(torch.complex64)[None, :]
    want = np.zeros((1, n), np.complex128)
    want[0, m] = n
    got = to_np(run(tone))
    assert np.max(np.abs(got - want)) <= 1e-5 * n


@pytest.mark.parametrize("n", [2, 16, 32, 256, 512, 2048])
def test_in_place(n):
    x = synth.uniform(301, n, seed=9)
    y = run(x, inplace=True)
    assert max_rel_l2(to_np(y), oracle_of(x)) <= FP32_TOL


@pytest.mark.parametrize("batch", [0, 1, 2, 31, 33])
@pytest.mark.parametrize("n", [2, 8, 64, 1024, 2048])
def test_small_and_empty_batches(n, batch):
    x = synth.uniform(batch, n, seed=11)
    y = run(x)
    assert y.shape == (batch, n)
    if batch:
        assert max_rel_l2(to_np(y), oracle_of(x)) <= FP32_TOL


def test_rejects_misaligned_and_overlapping():
    n, batch = 64, 8
    buf = torch.zeros(batch * n + 4, dtype=torch.complex64, device="cuda")
    plan = gb.Plan(n, batch)
    L = _abi.lib()
    base = buf.data_ptr()
    # 8-byte offset: complex64 aligned but not 16-byte aligned
    assert L.fft_execute(plan.handle, base + 8, base + 8 * (batch * n + 2), None) == \
        _abi.STATUS_CODE["FFT_ERR_MISALIGNED"]
    # aligned but partially overlapping ranges
    assert L.fft_execute(plan.handle, base, base + 16, None) == _abi.STATUS_CODE["FFT_ERR_OVERLAP"]
    assert L.fft_execute(plan.handle, None, base, None) == _abi.STATUS_CODE["FFT_ERR_INVALID_VALUE"]
    torch.cuda.synchronize()
    # the binding checks what the bare pointers cannot carry: size, dtype, device
    x = torch.zeros(batch, n, dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError):
        plan.execute(x, torch.empty(batch * n - 1, dtype=torch.complex64, device="cuda"))
    with pytest.raises(ValueError):
        plan.execute(x, torch.empty(batch, n, dtype=torch.complex64))
    with pytest.raises(ValueError):
        plan.execute(x.cpu())
    with pytest.raises(TypeError):
        plan.execute(x.to(torch.complex128))
    plan.close()


def test_plan_info_and_device_twiddles():
    for n in POW2:
        plan = gb.Plan(n, 1000)
        info = plan.info()
        assert info.n == n and info.batch == 1000 and info.grid >= 1
        prod = 1
        for s in range(info.num_stages):
            prod *= info.radix[s]
        assert prod == n
        cnt = info.twiddle_count
        if cnt:
            host = (ctypes.c_float * (2 * cnt))()
            assert _abi.lib().fft_plan_get_twiddles(plan.handle, host, cnt) == 0
            tw = np.frombuffer(host, dtype=np.float32).astype(np.float64)
            z = tw[0::2] + 1j * tw[1::2]
            assert np.allclose(np.abs(z), 1.0, atol=1e-7)
        plan.close()


def test_graph_capture_and_streams():
    n, batch = 1024, 4099
    x = synth.uniform(batch, n, seed=21).cuda()
    out = torch.empty_like(x)
    plan = gb.Plan(n, batch)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.execute(x, out)  # warm-up on a side stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(g):
        plan.execute(x, out)
    g.replay()
    torch.cuda.synchronize()
    ref = oracle_of(x.cpu())
    assert max_rel_l2(to_np(out), ref) <= FP32_TOL
    plan.close()


def test_variant_selection():
    for n in POW2:
        count = gb.fft_variant_count(n)
        assert count >= 1
        for v in range(count):
            dt = gb.DTYPE_NAMES[gb.fft_variant_dtype(n, v)]
            p = gb.Plan(n, 64, variant=v, dtype=dt)
            assert p.info().variant == v
            p.close()
            if dt != "c64":  # a tensor-core or complex32 variant is refused for FP32 plans
                with pytest.raises(gb.FFTError):
                    gb.Plan(n, 64, variant=v)
        with pytest.raises(gb.FFTError):
            gb.Plan(n, 64, variant=count)
    assert gb.fft_variant_count(12) == 0


FULL_BATCH_LENGTHS = (256, 2048)


@pytest.mark.parametrize("n", POW2)
def test_full_size(n):
    """The benchmark's workload: N * batch = 2^28 complex64 (2 GiB in), U[-1,1]
    drawn on the device from seed 1, launched exactly as the benchmark
    launches it.  For N = 256 and N = 2048 EVERY signal of the batch is
    compared element by element with the FP64 oracle (a chunk of 2^24
    elements at a time); for the other lengths a seeded set of 4096 signals
    (the first, the last and random ones).  As a cheap extra, every signal of
    every length is also checked against Parseval and the bins 0 and N/2."""
    batch = 2 ** 28 // n
    x = synth.uniform(batch, n, seed=1, device="cuda")
    out = torch.empty_like(x)
    plan = gb.Plan(n, batch)
    plan.execute(x, out)
    torch.cuda.synchronize()
    assert plan.error() == 0
    plan.close()
    if n in FULL_BATCH_LENGTHS:
        rows = None
    else:
        rng = np.random.default_rng(n)
        rows = np.unique(np.concatenate([[0, 1, batch - 1], rng.choice(batch, 4096 - 3, replace=False)]))
        assert rows.size >= 4096
    err, where = oracle_max_rel_l2(x, out, rows=rows)
    assert err <= FP32_TOL, (n, err, where)
    bad = every_signal_violations(x, out, FP32_TOL)
    assert bad.numel() == 0, bad[:8]
    del x, out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [16, 2048])
def test_beyond_2_32_elements(n):
    """One call over more than 2^32 complex64 elements (34 GB in, 34 GB out):
    64-bit signal and element indexing in every kernel of the length; the
    signals on both sides of element 2^32 and the last ones are checked against
    the oracle, every signal against Parseval and the bins 0 and N/2."""
    batch = (2 ** 32) // n + 3
    if torch.cuda.mem_get_info()[0] < 2 * 8 * n * batch + (4 << 30):
        pytest.skip("needs about 70 GB of free device memory")
    x = torch.empty(batch, n, dtype=torch.complex64, device="cuda")
    torch.view_as_real(x).uniform_(-1.0, 1.0, generator=torch.Generator(device="cuda").manual_seed(7))
    out = torch.empty_like(x)
    plan = gb.Plan(n, batch)
    plan.execute(x, out)
    torch.cuda.synchronize()
    assert plan.error() == 0
    plan.close()
    first_hi = (2 ** 32) // n  # first signal at or past element 2^32
    idx = np.unique(np.concatenate([[0], np.arange(first_hi - 3, batch)]))
    ti = torch.from_numpy(idx).cuda()
    xs = x.index_select(0, ti).cpu()
    ys = to_np(out.index_select(0, ti))
    bad = every_signal_violations(x, out, FP32_TOL)
    del x, out
    torch.cuda.empty_cache()
    assert bad.numel() == 0, bad[:8]
    assert max_rel_l2(ys, oracle_of(xs)) <= FP32_TOL


@pytest.mark.parametrize("n,batch", [(2, 70001), (64, 3 * 2 ** 20 // 64 + 5), (2048, 9001), (256, 1)])
def test_execute_host_pipeline(n, batch):
    """fft_execute_host: pinned host buffers, chunked copy / transform / copy
    over the plan's streams; chunk tails and single-chunk batches."""
    x = synth.uniform(batch, n, seed=41).pin_memory()
    plan = gb.Plan(n, batch, host_staging=True)
    y = plan.execute_host(x)
    assert plan.error() == 0
    rng = np.random.default_rng(n)
    idx = np.unique(np.concatenate([[0, batch - 1], rng.integers(0, batch, 300)]))
    assert max_rel_l2(y.numpy()[idx], oracle_of(x[idx])) <= FP32_TOL
    # in place on the host
    z = x.clone().pin_memory()
    plan.execute_host(z, z)
    assert torch.equal(z, y)
    plan.close()
    # a plan made without staging refuses host execution
    p2 = gb.Plan(n, batch)
    with pytest.raises(gb.FFTError):
        p2.execute_host(x)
    p2.close()
