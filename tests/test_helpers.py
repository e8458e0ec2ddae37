"""CPU checks of the test helpers themselves: the every-signal property check
must pass exact transforms and flag planted mistakes."""
import numpy as np
import torch

import oracle
import synth
from tests.helpers import every_signal_violations, oracle_max_rel_l2


def test_every_signal_check_passes_the_oracle_and_flags_mistakes():
    n, batch = 64, 300
    x = synth.uniform(batch, n, seed=5)
    y = torch.from_numpy(oracle.reference(x.numpy().astype(np.complex128), threads=2))
    assert every_signal_violations(x, y, 1e-5).numel() == 0
    assert every_signal_violations(x, y.to(torch.complex64), 1e-5, chunk_elems=1000).numel() == 0
    bad = y.clone()
    bad[3] *= 1.001          # wrong scale (Parseval)
    bad[40] = bad[41]        # another signal's output (bin 0)
    bad[100, n // 2] *= -1   # sign of the Nyquist bin
    bad[batch - 1] = 0       # a signal never written
    got = every_signal_violations(x, bad, 1e-5, chunk_elems=1000)
    assert got.tolist() == [3, 40, 100, batch - 1]


def test_every_signal_check_zero_signals_and_length_two():
    z = torch.zeros(4, 8, dtype=torch.complex64)
    assert every_signal_violations(z, z, 1e-5).numel() == 0
    off = z.clone()
    off[2, 1] = 1e-3         # zero input: the bar is absolute
    assert every_signal_violations(z, off, 1e-5).tolist() == [2]
    x = synth.uniform(5, 2, seed=6)
    y = torch.stack([x[:, 0] + x[:, 1], x[:, 0] - x[:, 1]], dim=1)
    assert every_signal_violations(x, y, 1e-5).numel() == 0


def test_oracle_comparison_covers_every_signal_and_finds_a_planted_mistake():
    """oracle_max_rel_l2 compares signal by signal with the oracle: numpy's FFT
    (an independent library) of the same inputs passes near FP64 rounding, and
    a single wrong bin, a permutation of two bins or one signal copied over
    another is found at its own index, whatever chunk it falls in."""
    n, batch = 128, 301
    x = synth.uniform(batch, n, seed=8)
    y = torch.from_numpy(np.fft.fft(x.numpy().astype(np.complex128), axis=1))
    err, _ = oracle_max_rel_l2(x, y, chunk_elems=50 * n, threads=2)
    assert err < 1e-13
    for planted in (7, 149, batch - 1):
        bad = y.clone()
        bad[planted, 5] += 1e-3 * torch.linalg.vector_norm(bad[planted])
        err, where = oracle_max_rel_l2(x, bad, chunk_elems=50 * n, threads=2)
        assert where == planted and 0.9e-3 < err < 1.1e-3
    swapped = y.clone()
    swapped[60, [3, 4]] = swapped[60, [4, 3]]  # keeps Parseval and the bins 0 and N/2
    assert every_signal_violations(x, swapped, 1e-5).numel() == 0
    err, where = oracle_max_rel_l2(x, swapped, chunk_elems=50 * n, threads=2)
    assert where == 60 and err > 1e-3
    # a subset of rows, given as indices; the inverse direction
    rows = np.array([0, 60, 299])
    err, where = oracle_max_rel_l2(x, swapped, rows=rows, chunk_elems=2 * n, threads=2)
    assert where == 60
    xi = torch.from_numpy(np.fft.ifft(x.numpy().astype(np.complex128), axis=1))
    err, _ = oracle_max_rel_l2(x, xi, inverse=True, threads=2)
    assert err < 1e-13
