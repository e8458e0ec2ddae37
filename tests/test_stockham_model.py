"""The generic kernels' Stockham index mapping, replayed on the CPU (no GPU).

For every schedule row of csrc/schedules.h (FP32, tensor-core and complex32
rows share the mapping), one tile of S signals goes through the kernels'
index arithmetic in numpy: the stage-0 load (``load_first`` for direct
kernels, ``gather_tile`` for the bulk-copy ring), per stage the twiddle
omega_{Ns R}^{(j mod Ns) r} at table entry tw_off(s) + (r-1) Ns + (j mod Ns)
and an exact R-point DFT, the ``scatter``/``gather`` exchanges through the
8-byte XOR swizzle, and ``store_last``.  The result must be the DFT of each
signal (Eq. (dft); numpy's FFT as the library reference), every exchange
slot must be written once per stage and never read before it is written.
A schedule row with a wrong radix split, thread mapping or stride fails here
before it reaches a GPU.
"""
import numpy as np
import pytest

from tests.test_bank_model import _rows, swz8


def all_rows():
    rows = []
    for L, v, E, S, r0, r1, r2, r3, minb, pipe, tc, xb, ch in _rows("GBFFT_GENERIC_SCHEDULES", 13):
        kind = "GX-shuffle" if xb == 3 else "GX-padded" if xb == -5 else "GX"
        rows.append((kind, L, v, E, S, [r for r in (r0, r1, r2, r3) if r], pipe))
    for L, v, E, S, r0, r1, r2, r3, minb, pipe, xb in _rows("GBFFT_C32_SCHEDULES", 11):
        rows.append(("CX", L, v, E, S, [r for r in (r0, r1, r2, r3) if r], pipe))
    return rows


def shuffle_transpose(v, plant=None):
    """The kernels' shuffle_transpose on the registers of one signal's R
    lanes: v[t, q] (lane t, register q) for an R x R tile.  For each lane bit
    b, lanes t and t ^ b exchange: the lane with bit b clear sends v[q | b]
    and keeps v[q], the other sends v[q] and keeps v[q | b] (q with bit b
    clear).  Returns the registers after all rounds."""
    R = v.shape[0]
    v = v.copy()
    b = R // 2
    while b >= 1:
        send = np.empty_like(v)
        for t in range(R):
            hi = bool(t & b) if plant != "lane-bit" else bool(t & (b >> 1 or R // 2))
            for q in range(R):
                if q & b:
                    continue
                send[t, q] = v[t, q] if hi else v[t, q | b]
        for t in range(R):
            hi = bool(t & b) if plant != "lane-bit" else bool(t & (b >> 1 or R // 2))
            for q in range(R):
                if q & b:
                    continue
                got = send[t ^ b, q]  # __shfl_xor_sync(send, b)
                if hi:
                    v[t, q] = got
                else:
                    v[t, q | b] = got
        b //= 2
    return v


def replay(N, E, S, radix, pipe, x, plant=None, shuffle=False, pad=0):
    """x: [S, N] complex; returns the tile's output [S, N] as the kernel
    computes it (exact arithmetic in complex128).  `plant` puts one plausible
    mistake into the mapping, to show the replay can fail.  `pad`: the ring
    slot holds signal q at element q (N + pad), as the per-signal copies of a
    padded in-ring schedule write it (XB = -5), and stage 0 reads it there."""
    T = N // E
    NT = T * S
    M = len(radix)

    def ns(s):
        return int(np.prod(radix[:s], dtype=np.int64)) if s else 1

    def bfly(s, t, c):
        K = E // radix[s]
        if (s == 0 and pipe == 0) or s == M - 1:
            return K * t + c
        return t + T * c

    flat = np.full(S * (N + pad), np.nan + 0j)  # the slot as the copies write it
    for q in range(S):
        flat[q * (N + pad):q * (N + pad) + N] = x[q]
    v = np.zeros((NT, E), dtype=np.complex128)
    R, K, stride = radix[0], E // radix[0], N // radix[0]
    for tid in range(NT):
        sb, t = (tid // T) * (N + pad), tid % T
        for c in range(K):
            j = bfly(0, t, c)
            for r in range(R):
                v[tid, c * R + r] = flat[sb + j + r * stride]
    for s in range(M):
        R, K, Ns = radix[s], E // radix[s], ns(s)
        if s > 0 and shuffle:
            # the warp-shuffle exchange of a two-stage R x R schedule
            assert M == 2 and radix[0] == radix[1] == E == T
            for g in range(NT // T):
                v[g * T:(g + 1) * T] = shuffle_transpose(v[g * T:(g + 1) * T], plant)
        elif s > 0:
            # exchange: scatter stage s-1's outputs, gather stage s's inputs
            Rp, Kp, Nsp = radix[s - 1], E // radix[s - 1], ns(s - 1)
            buf = {}
            for tid in range(NT):
                sb, t = (tid // T) * N, tid % T
                for c in range(Kp):
                    j = bfly(s - 1, t, c)
                    base = sb + (j // Nsp) * (Nsp * Rp) + (j % Nsp)
                    for q in range(Rp):
                        a = swz8(base + q * Nsp, N)
                        if plant == "scatter":  # written with the read pattern
                            a = swz8(sb + j + q * (N // Rp), N)
                        assert a not in buf, f"stage {s}: slot {a} written twice"
                        assert 0 <= a < S * N, f"stage {s}: slot {a} outside the tile"
                        buf[a] = v[tid, c * Rp + q]
            stride = N // R + (1 if plant == "stride" else 0)
            for tid in range(NT):
                sb, t = (tid // T) * N, tid % T
                for c in range(K):
                    j = bfly(s, t, c)
                    for r in range(R):
                        a = swz8(sb + j + r * stride, N)
                        assert a in buf, f"stage {s}: slot {a} read before it is written"
                        v[tid, c * R + r] = buf[a]
        w = np.exp(-2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
        for tid in range(NT):
            t = tid % T
            for c in range(K):
                seg = v[tid, c * R:(c + 1) * R]
                if s > 0:
                    j = bfly(s, t, c)
                    sign = 1 if plant == "twiddle" else -1
                    seg = seg * np.exp(sign * 2j * np.pi * ((j % Ns) * np.arange(R)) / (Ns * R))
                v[tid, c * R:(c + 1) * R] = w @ seg
    out = np.full(S * N, np.nan + 0j)
    R, K, stride = radix[M - 1], E // radix[M - 1], N // radix[M - 1]
    for tid in range(NT):
        sb, t = (tid // T) * N, tid % T
        for c in range(K):
            j = bfly(M - 1, t, c)
            for q in range(R):
                out[sb + j + q * stride] = v[tid, c * R + q]
    return out.reshape(S, N)


@pytest.mark.parametrize("row", all_rows(), ids=lambda r: f"{r[0]}-N{1 << r[1]}-v{r[2]}")
def test_schedule_row_computes_the_dft(row):
    kind, L, variant, E, S, radix, pipe = row
    N = 1 << L
    assert int(np.prod(radix)) == N and all(E % r == 0 for r in radix)
    rng = np.random.default_rng(L * 100 + variant)
    x = rng.standard_normal((S, N)) + 1j * rng.standard_normal((S, N))
    y = replay(N, E, S, radix, pipe, x, shuffle=kind == "GX-shuffle", pad=N // E if kind == "GX-padded" else 0)
    assert not np.isnan(y).any(), "an output element was never stored"
    assert np.allclose(y, np.fft.fft(x, axis=1), rtol=0, atol=1e-9 * N)


@pytest.mark.parametrize("plant", ["twiddle", "scatter", "stride"])
def test_replay_fails_on_a_planted_mistake(plant):
    """A twiddle sign, a Stockham write in the read pattern or a gather
    stride off by one must not pass for the N = 64, 1024 and 2048 defaults."""
    for n, E, S, radix, pipe in ((64, 16, 64, [8, 8], 0), (1024, 16, 2, [8, 16, 8], 2),
                                 (2048, 16, 1, [8, 16, 16], 2)):
        rng = np.random.default_rng(n)
        x = rng.standard_normal((S, n)) + 1j * rng.standard_normal((S, n))
        assert np.allclose(replay(n, E, S, radix, pipe, x), np.fft.fft(x, axis=1), atol=1e-9 * n)
        try:
            y = replay(n, E, S, radix, pipe, x, plant=plant)
            ok = not np.isnan(y).any() and np.allclose(y, np.fft.fft(x, axis=1), atol=1e-9 * n)
        except AssertionError:
            ok = False
        assert not ok, (plant, n)


@pytest.mark.parametrize("R", [2, 4, 8, 16, 32])
def test_shuffle_transpose_is_the_stockham_read(R):
    """The shuffle rounds leave lane t holding column t (v[t, r] = in[r, t]),
    which is the read y[t + R r] of the second stage; a lane bit taken from
    the wrong round breaks it."""
    rng = np.random.default_rng(R)
    m = rng.standard_normal((R, R)) + 1j * rng.standard_normal((R, R))
    assert np.array_equal(shuffle_transpose(m), m.T)
    if R >= 4:
        assert not np.array_equal(shuffle_transpose(m, plant="lane-bit"), m.T)
