"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, validates arguments, and builds an exact twiddle table."""
import ctypes
import math
import subprocess

import numpy as np
import pytest
import torch

from paper_2203_09384_gb300 import _abi


@pytest.fixture(scope="module")
def L():
    return _abi.lib()


def test_exports_every_declared_symbol(L):
    declared = _abi.declared_symbols()
    assert "fft_plan_create" in declared and "fft_execute" in declared and "fft_plan_destroy" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(L, s)


def test_status_strings(L):
    for code in _abi.STATUS:
        assert L.fft_status_string(code)
    assert L.fft_status_string(999) == b"unknown status"


@pytest.mark.parametrize("n", [0, 1, 3, 6, 12, 100, 4096, 2 ** 20, -8])
def test_invalid_sizes(n):
    assert _abi.fft_validate(n, 1) == _abi.STATUS_CODE["FFT_ERR_INVALID_SIZE"]
    with pytest.raises(_abi.FFTError) as e:
        _abi.fft_plan_create(n, 1)
    assert e.value.name == "FFT_ERR_INVALID_SIZE"


def test_invalid_values():
    bad = _abi.STATUS_CODE["FFT_ERR_INVALID_VALUE"]
    assert _abi.fft_validate(64, -1) == bad
    assert _abi.fft_validate(64, 1, direction=2) == bad
    assert _abi.fft_validate(64, 1, direction=-1) == bad
    assert _abi.fft_validate(64, 1, dtype=7) == bad
    assert _abi.fft_validate(64, 1, flags=1 << 20) == bad
    assert _abi.fft_validate(2048, 2 ** 62) == bad  # byte count overflows


def test_valid_arguments():
    for k in range(1, 12):
        assert _abi.fft_validate(2 ** k, 0) == 0
        assert _abi.fft_validate(2 ** k, 3, 1, 0, _abi.FFT_FLAG_UNNORMALIZED) == 0
        assert _abi.fft_validate(2 ** k, 3, 0, _abi.FFT_C32) == 0


def test_complex32_registry():
    """Each length has complex32-storage variants; they are refused as the
    default of the complex64 path and with host staging."""
    for k in range(1, 12):
        n = 2 ** k
        kinds = [_abi.lib().fft_variant_dtype(n, v) for v in range(_abi.fft_variant_count(n))]
        assert kinds.count(_abi.FFT_C32) >= 1
        assert kinds[_abi.fft_get_default_variant(n)] == _abi.FFT_C64
    assert _abi.fft_validate(64, 1, 0, _abi.FFT_C32, _abi.FFT_FLAG_HOST_STAGING) == \
        _abi.STATUS_CODE["FFT_ERR_UNSUPPORTED"]
    assert _abi.fft_validate(64, 1, dtype=4) == _abi.STATUS_CODE["FFT_ERR_INVALID_VALUE"]


def test_null_arguments(L):
    assert L.fft_plan_create(64, 1, 0, 0, None) == _abi.STATUS_CODE["FFT_ERR_INVALID_VALUE"]
    assert L.fft_execute(None, None, None, None) == _abi.STATUS_CODE["FFT_ERR_INVALID_VALUE"]
    assert L.fft_plan_destroy(None) == 0
    assert L.fft_plan_get_info(None, None) == _abi.STATUS_CODE["FFT_ERR_INVALID_VALUE"]


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU path")
def test_no_device_reported():
    with pytest.raises(_abi.FFTError) as e:
        _abi.fft_plan_create(64, 4)
    assert e.value.name == "FFT_ERR_NO_DEVICE"


def _fp32_round(z):
    return complex(np.float32(z.real), np.float32(z.imag))


@pytest.mark.parametrize("m", [2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 3, 6, 12])
def test_twiddles_are_correctly_rounded(m):
    """Each FP32 twiddle is within half an ulp of exp(-2 pi i k/m) (FP64)."""
    for k in range(m):
        got = _abi.fft_twiddle_fp32(m, k)
        exact = complex(math.cos(2 * math.pi * k / m), -math.sin(2 * math.pi * k / m))
        for g, e in ((got.real, exact.real), (got.imag, exact.imag)):
            ulp = np.spacing(np.float32(abs(e))) if e != 0 else np.float32(1e-45)
            assert abs(g - e) <= 0.5 * ulp + 2e-16, (m, k, got, exact)


@pytest.mark.parametrize("m", [4, 8, 16, 64, 256, 2048])
def test_twiddle_symmetry_is_exact(m):
    """Sec. 3.1, Eq. (twiddle): omega^{k+m/4} = -i omega^k, bit for bit in FP32,
    and the quadrant points 1, -i, -1, i are exact."""
    for k in range(m):
        a = _abi.fft_twiddle_fp32(m, k)
        b = _abi.fft_twiddle_fp32(m, k + m // 4)
        assert b == complex(a.imag, -a.real) or (b.real == a.imag and b.imag == -a.real)
        c = _abi.fft_twiddle_fp32(m, k + m)  # periodicity
        assert c == a
    assert _abi.fft_twiddle_fp32(m, 0) == 1
    assert _abi.fft_twiddle_fp32(m, m // 4) == -1j
    assert _abi.fft_twiddle_fp32(m, m // 2) == -1
    assert _abi.fft_twiddle_fp32(m, 3 * m // 4) == 1j


def test_header_has_no_torch_types():
    with open(_abi.HEADER) as f:
        text = f.read()
    assert "torch" not in text.lower().replace("pytorch", "") or "at::" not in text
    assert "at::Tensor" not in text and "c10" not in text


def test_schedule_variant_numbers_are_unique():
    """Every (length, variant) pair names ONE row across the four schedule
    tables (FP32/tensor-core, one-thread-per-signal, complex32 and its
    one-thread-per-signal form): a duplicate would silently replace a row in
    the registry.  Each row's variant is in the flag's range, and the library
    reports each row with the dtype of its own table."""
    from tests.test_bank_model import _rows

    seen = {}
    tables = [("GBFFT_GENERIC_SCHEDULES", 13), ("GBFFT_SMALL_SCHEDULES", 5),
              ("GBFFT_C32_SCHEDULES", 11), ("GBFFT_C32_SMALL_SCHEDULES", 5)]
    for macro, nargs in tables:
        rows = _rows(macro, nargs)
        assert rows, macro
        for row in rows:
            key = (row[0], row[1])
            assert key not in seen, f"variant {row[1]} of N=2^{row[0]} in {macro} and {seen.get(key)}"
            seen[key] = macro
            assert 0 <= row[1] <= 30
            want = {"GBFFT_C32_SCHEDULES": _abi.FFT_C32, "GBFFT_C32_SMALL_SCHEDULES": _abi.FFT_C32,
                    "GBFFT_SMALL_SCHEDULES": _abi.FFT_C64}.get(macro)
            if want is None:  # generic rows: the TC column picks the dtype
                want = [_abi.FFT_C64, _abi.FFT_C64_TC_F16, _abi.FFT_C64_TC_BF16][row[10] & 3]
            assert _abi.fft_variant_dtype(2 ** row[0], row[1]) == want, (macro, row)
    for k in range(1, 12):
        used = {v for (L, v) in seen if L == k}
        assert _abi.fft_variant_count(2 ** k) == max(used) + 1
        assert used == set(range(max(used) + 1)), f"N=2^{k}: variant numbers with no row"
