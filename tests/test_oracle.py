"""The FP64 oracle against its pins, and the pins against planted mistakes.

CPU only (no GPU marker): these run under ``-m "not gpu"``.
"""
import numpy as np
import pytest

import oracle
from tests import oracle_pins as pins


@pytest.fixture(scope="module")
def orc():
    return oracle.Oracle(0)


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(orc, pin):
    pin(orc)


@pytest.mark.parametrize("mutant", sorted(oracle.MUTANTS))
def test_planted_mistake_is_caught(mutant):
    """Each planted mistake in the oracle must fail at least one pin."""
    bad = oracle.Oracle(mutant)
    failed = []
    for pin in pins.ALL_PINS:
        try:
            pin(bad)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {mutant} ({oracle.MUTANTS[mutant]}) passed every pin"


def test_threads_do_not_change_results(orc):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((37, 128)) + 1j * rng.standard_normal((37, 128))
    a = orc.fft_radix2(x, threads=1)
    b = orc.fft_radix2(x, threads=5)
    assert np.array_equal(a, b)


def test_rejects_bad_arguments(orc):
    with pytest.raises(ValueError):
        orc.fft_radix2(np.zeros((1, 12), np.complex128))


def test_empty_batch(orc):
    y = orc.fft_radix2(np.zeros((0, 64), np.complex128))
    assert y.shape == (0, 64)
