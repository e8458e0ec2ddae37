"""CPU checks of the test helpers themselves: the every-signal property check
must pass exact transforms and flag planted mistakes."""
import numpy as np
import torch

import oracle
import synth
from tests.helpers import every_signal_violations


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
