"""Pins for the FP64 oracle: facts fixed by the paper and by mathematics.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError when the
oracle disagrees with something other than itself: hand-evaluated values,
closed forms, theorems of the DFT, the identities of Sec. 3.1 rebuilt from
smaller transforms, an independent library FFT (numpy's pocketfft, used only
here) and finite differences.  The set is chosen so that every planted
mistake in ``oracle.MUTANTS`` fails at least one pin (checked by a test).
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_exact.txt")
POW2 = [2 ** k for k in range(1, 12)]
TOL = 1e-11  # FP64 relative L2, well above the ~N*u error of either routine


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    d = np.linalg.norm((a - b).ravel())
    r = np.linalg.norm(b.ravel())
    return d / r if r > 0 else d


def both(orc, x, inverse=False, normalize=True):
    """Run the naive and the recursive routine where both apply."""
    n = np.asarray(x).shape[-1]
    outs = [orc.fft_radix2(x, inverse, normalize)]
    if n <= 256:
        outs.append(orc.dft_naive(x, inverse, normalize))
    return outs


def _parse(field):
    vals = []
    for pair in field.split(";"):
        re_, im_ = pair.split(",")
        vals.append(complex(float(re_), float(im_)))
    return np.array(vals, dtype=np.complex128)


def golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, xin, xout = [p.strip() for p in line.split("|")]
            direction, n = head.split()
            rows.append((direction == "inverse", int(n), _parse(xin), _parse(xout)))
    return rows


def pin_golden_small(orc):
    for inverse, n, x, y in golden_rows():
        assert x.size == n and y.size == n
        for out in (orc.dft_naive(x, inverse), orc.fft_radix2(x, inverse)):
            assert np.max(np.abs(out - y)) < 1e-13, (inverse, n, out, y)


def _root_powers(n, e):
    """omega_N^e for integer array e, the exponent reduced mod N first."""
    m = np.mod(e, n).astype(np.float64)
    return np.exp(-2j * np.pi * m / n)


def pin_delta(orc):
    for n in POW2:
        for n0 in sorted({0, 1, n // 2, n - 1}):
            x = np.zeros(n, np.complex128)
            x[n0] = 1.0
            want = _root_powers(n, np.arange(n) * n0)  # X_k = omega^{k n0}
            for out in both(orc, x):
                assert rel_l2(out, want) < TOL, (n, n0)


def pin_single_tone(orc):
    for n in POW2:
        for m in sorted({0, 1, n // 3, n - 1}):
            x = np.conj(_root_powers(n, np.arange(n) * m))  # omega^{-mn}
            want = np.zeros(n, np.complex128)
            want[m] = n
            for out in both(orc, x):
                assert np.max(np.abs(out - want)) < 1e-9 * n, (n, m)
            # inverse maps the spike back to the tone
            back = orc.fft_radix2(want, inverse=True)
            assert rel_l2(back, x) < TOL


def ramp_closed_form(n, inverse=False):
    """DFT of x_k = k (the paper's f(x) = x): X_0 = N(N-1)/2 and, for k != 0,
    X_k = N/(omega^k - 1) = -N/2 + i (N/2) cot(pi k / N).  The inverse
    (Eq. (idft), with 1/N) is the conjugate divided by N."""
    k = np.arange(n)
    out = np.empty(n, np.complex128)
    out[0] = n * (n - 1) / 2.0
    kk = k[1:]
    out[1:] = -n / 2.0 + 1j * (n / 2.0) / np.tan(np.pi * kk / n)
    if inverse:
        out = np.conj(out) / n
    return out


def pin_ramp(orc):
    for n in POW2:
        x = np.arange(n, dtype=np.float64).astype(np.complex128)
        for inverse in (False, True):
            want = ramp_closed_form(n, inverse)
            for out in both(orc, x, inverse):
                assert rel_l2(out, want) < TOL, (n, inverse)


def _rng(seed):
    return np.random.default_rng(seed)


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def pin_linearity(orc):
    rng = _rng(11)
    for n in POW2:
        a, b = _crandn(rng, 2, n)
        alpha, beta = 0.75 - 0.5j, -1.25 + 2.0j
        lhs = orc.fft_radix2(alpha * a + beta * b)
        rhs = alpha * orc.fft_radix2(a) + beta * orc.fft_radix2(b)
        assert rel_l2(lhs, rhs) < TOL, n


def pin_parseval(orc):
    rng = _rng(12)
    for n in POW2:
        x = _crandn(rng, 3, n)
        for out in both(orc, x):
            lhs = np.sum(np.abs(out) ** 2, axis=1)
            rhs = n * np.sum(np.abs(x) ** 2, axis=1)
            assert np.max(np.abs(lhs - rhs) / rhs) < TOL, n


def pin_round_trip(orc):
    rng = _rng(13)
    for n in POW2:
        x = _crandn(rng, 2, n)
        y = orc.fft_radix2(orc.fft_radix2(x), inverse=True)
        assert rel_l2(y, x) < TOL, n
        if n <= 256:
            z = orc.dft_naive(orc.dft_naive(x), inverse=True)
            assert rel_l2(z, x) < TOL, n
        # the unnormalised inverse is exactly N times the normalised one
        u = orc.fft_radix2(x, inverse=True, normalize=False)
        v = orc.fft_radix2(x, inverse=True, normalize=True)
        assert rel_l2(u, n * v) < TOL, n


def pin_naive_equals_recursive(orc):
    """Brute force: the O(N^2) sum and the recursion agree on every N <= 64
    and on every basis vector at N <= 16."""
    rng = _rng(14)
    for n in [2, 4, 8, 16, 32, 64]:
        x = _crandn(rng, 4, n)
        for inverse in (False, True):
            a = orc.dft_naive(x, inverse)
            b = orc.fft_radix2(x, inverse)
            assert rel_l2(a, b) < 1e-13, (n, inverse)
        if n <= 16:
            eye = np.eye(n, dtype=np.complex128)
            assert rel_l2(orc.dft_naive(eye), orc.fft_radix2(eye)) < 1e-13


def pin_library(orc):
    """numpy's pocketfft (FP64) as an independent third opinion."""
    rng = _rng(15)
    for n in POW2:
        x = _crandn(rng, 3, n)
        assert rel_l2(orc.fft_radix2(x), np.fft.fft(x, axis=1)) < TOL, n
        assert rel_l2(orc.fft_radix2(x, inverse=True), np.fft.ifft(x, axis=1)) < TOL, n
        if n <= 256:
            assert rel_l2(orc.dft_naive(x), np.fft.fft(x, axis=1)) < TOL, n


def pin_shift_and_modulation(orc):
    rng = _rng(16)
    for n in POW2:
        x = _crandn(rng, n)
        s = n // 2 + 1 if n > 2 else 1
        X = orc.fft_radix2(x)
        # time shift: x_{(t - s) mod N} -> X_k omega^{k s}
        shifted = orc.fft_radix2(np.roll(x, s))
        assert rel_l2(shifted, X * _root_powers(n, np.arange(n) * s)) < TOL, n
        # modulation: x_t omega^{-m t} -> X_{(k - m) mod N}
        m = 1
        mod = orc.fft_radix2(x * np.conj(_root_powers(n, np.arange(n) * m)))
        assert rel_l2(mod, np.roll(X, m)) < TOL, n


def pin_conjugate_symmetry(orc):
    rng = _rng(17)
    for n in POW2:
        x = rng.standard_normal(n).astype(np.complex128)
        for X in both(orc, x):
            k = np.arange(n)
            assert rel_l2(X[(n - k) % n], np.conj(X)) < TOL, n


def pin_radix2_identity(orc):
    """Eq. (radix2) rebuilt from two half-length DFTs of the naive routine."""
    rng = _rng(18)
    for n in [4, 8, 16, 32, 64, 128, 256]:
        x = _crandn(rng, n)
        E = orc.dft_naive(x[0::2])
        O = orc.dft_naive(x[1::2])
        w = _root_powers(n, np.arange(n // 2))
        want = np.concatenate([E + w * O, E - w * O])
        assert rel_l2(orc.fft_radix2(x), want) < TOL, n
        assert rel_l2(orc.dft_naive(x), want) < TOL, n


def pin_split_radix_identity(orc):
    """Sec. 3.1 split-radix, Eq. (split-radix-final): X_k = E_k + w^k O_k + w^{3k} O'_k and its three
    companions at k + N/4, k + N/2, k + 3N/4 (k < N/4), E the N/2-point DFT
    of the even samples, O / O' the N/4-point DFTs of samples 4n+1 / 4n+3."""
    rng = _rng(19)
    for n in [4, 8, 16, 32, 64, 128, 256, 512]:
        x = _crandn(rng, n)
        E = orc.fft_radix2(x[0::2])
        O = orc.fft_radix2(x[1::4])
        O3 = orc.fft_radix2(x[3::4])
        q = n // 4
        k = np.arange(q)
        a = _root_powers(n, k) * O
        b = _root_powers(n, 3 * k) * O3
        want = np.empty(n, np.complex128)
        want[k] = E[k] + (a + b)
        want[k + n // 2] = E[k] - (a + b)
        want[k + q] = E[k + q] - 1j * (a - b)
        want[k + 3 * q] = E[k + q] + 1j * (a - b)
        for out in both(orc, x):
            assert rel_l2(out, want) < TOL, n


def _loss(orc, x, w):
    X = orc.dft_naive(x) if x.shape[-1] <= 64 else orc.fft_radix2(x)
    return float(np.sum(np.abs(w * X) ** 2))


def pin_gradient_finite_difference(orc):
    """L(x) = sum |W * DFT(x)|^2 is quadratic, so the central difference is
    exact up to rounding; grad = dL/dRe + i dL/dIm."""
    rng = _rng(20)
    for n, batch in [(8, 2), (32, 1)]:
        x = _crandn(rng, batch, n)
        w = _crandn(rng, batch, n)
        g, L = orc.grad_weighted_power(x, w)
        assert abs(L - _loss(orc, x, w)) <= 1e-12 * abs(L)
        h = 1e-3
        fd = np.empty_like(x)
        for b in range(batch):
            for i in range(n):
                for unit, part in ((1.0, "re"), (1j, "im")):
                    xp = x.copy(); xp[b, i] += h * unit
                    xm = x.copy(); xm[b, i] -= h * unit
                    d = (_loss(orc, xp, w) - _loss(orc, xm, w)) / (2 * h)
                    if part == "re":
                        fd[b, i] = d
                    else:
                        fd[b, i] += 1j * d
        assert rel_l2(g, fd) < 1e-8, (n, rel_l2(g, fd))


def pin_gradient_euler(orc):
    """Euler's theorem for a degree-2 form: L = Re<grad, x> / 2."""
    rng = _rng(21)
    for n in [16, 256, 2048]:
        x = _crandn(rng, 2, n)
        w = _crandn(rng, 2, n)
        g, L = orc.grad_weighted_power(x, w)
        lhs = 0.5 * float(np.real(np.vdot(g, x)))
        assert abs(lhs - L) <= 1e-10 * abs(L), n


ALL_PINS = [
    pin_golden_small,
    pin_delta,
    pin_single_tone,
    pin_ramp,
    pin_linearity,
    pin_parseval,
    pin_round_trip,
    pin_naive_equals_recursive,
    pin_library,
    pin_shift_and_modulation,
    pin_conjugate_symmetry,
    pin_radix2_identity,
    pin_split_radix_identity,
    pin_gradient_finite_difference,
    pin_gradient_euler,
]
