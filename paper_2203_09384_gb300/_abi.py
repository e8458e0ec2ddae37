"""ctypes declarations for libgbfft.so (the C-ABI in include/gbfft.h).

Argument marshalling only.  The library is built in-tree into ``_build/``;
when it is missing this module raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgbfft.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gbfft.h")

FFT_FORWARD = 0
FFT_INVERSE = 1
FFT_C64 = 0
FFT_C64_TC_F16 = 1
FFT_C64_TC_BF16 = 2
FFT_C32 = 3
FFT_FLAG_UNNORMALIZED = 1 << 0
FFT_FLAG_SCALE_FORWARD = 1 << 1
FFT_FLAG_VARIANT_MASK = 0x1F << 8
FFT_FLAG_TEST_STALL = 1 << 16
FFT_FLAG_HOST_STAGING = 1 << 17


def FFT_FLAG_VARIANT(k: int) -> int:
    return (k + 1) << 8

STATUS = {
    0: "FFT_OK",
    1: "FFT_ERR_INVALID_SIZE",
    2: "FFT_ERR_INVALID_VALUE",
    3: "FFT_ERR_MISALIGNED",
    4: "FFT_ERR_OVERLAP",
    5: "FFT_ERR_ALLOC",
    6: "FFT_ERR_CUDA",
    7: "FFT_ERR_UNSUPPORTED",
    8: "FFT_ERR_TIMEOUT",
    9: "FFT_ERR_DEVICE_CHECK",
    10: "FFT_ERR_NO_DEVICE",
    11: "FFT_ERR_NOALLOC_LIMIT",
}
STATUS_CODE = {v: k for k, v in STATUS.items()}


class FFTError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        msg = f"{what}: {self.name}" if what else self.name
        try:
            msg += f" ({lib().fft_status_string(status).decode()})"
        except Exception:  # pragma: no cover - message only
            pass
        super().__init__(msg)


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("batch", ctypes.c_int64),
        ("direction", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("flags", ctypes.c_uint32),
        ("elems_per_thread", ctypes.c_int),
        ("signals_per_block", ctypes.c_int),
        ("threads_per_block", ctypes.c_int),
        ("num_stages", ctypes.c_int),
        ("radix", ctypes.c_int * 8),
        ("variant", ctypes.c_int),
        ("pipeline", ctypes.c_int),
        ("min_blocks", ctypes.c_int),
        ("kernel_kind", ctypes.c_int),
        ("work_items", ctypes.c_int64),
        ("tc", ctypes.c_int),
        ("grid", ctypes.c_int64),
        ("smem_bytes", ctypes.c_int64),
        ("twiddle_count", ctypes.c_int64),
        ("tc_stages", ctypes.c_int),
    ]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_u32 = ctypes.c_uint32


def declared_symbols() -> list[str]:
    """Every function the public header declares (GBFFT_API ... name(...))."""
    with open(HEADER) as f:
        text = f.read()
    return re.findall(r"GBFFT_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)


def lib() -> ctypes.CDLL:
    """Load libgbfft.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libgbfft.so not built ({LIB_PATH} missing); run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first")
    _lib = declare(ctypes.CDLL(LIB_PATH))
    return _lib


def declare(L: ctypes.CDLL) -> ctypes.CDLL:
    """Give every C-ABI entry point of a loaded build its ctypes signature
    (the package's own library, or the GBFFT_DEBUG build the tests load)."""
    L.fft_version.restype = ctypes.c_char_p
    L.fft_version.argtypes = []
    L.fft_status_string.restype = ctypes.c_char_p
    L.fft_status_string.argtypes = [_int]
    L.fft_validate.restype = _int
    L.fft_validate.argtypes = [_i64, _i64, _int, _int, _u32]
    L.fft_plan_create.restype = _int
    L.fft_plan_create.argtypes = [_i64, _i64, _int, _int, ctypes.POINTER(_vp)]
    L.fft_plan_create_ex.restype = _int
    L.fft_plan_create_ex.argtypes = [_i64, _i64, _int, _int, _u32, ctypes.POINTER(_vp)]
    L.fft_execute_c32.restype = _int
    L.fft_execute_c32.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.fft_execute_host.restype = _int
    L.fft_execute_host.argtypes = [_vp, _vp, _vp, _vp]
    L.fft_execute.restype = _int
    L.fft_execute.argtypes = [_vp, _vp, _vp, _vp]
    L.fft_plan_get_error.restype = _int
    L.fft_plan_get_error.argtypes = [_vp]
    L.fft_plan_destroy.restype = _int
    L.fft_plan_destroy.argtypes = [_vp]
    L.fft_plan_get_info.restype = _int
    L.fft_plan_get_info.argtypes = [_vp, ctypes.POINTER(PlanInfo)]
    L.fft_plan_get_twiddles.restype = _int
    L.fft_plan_get_twiddles.argtypes = [_vp, _vp, _i64]
    L.fft_variant_count.restype = _int
    L.fft_variant_count.argtypes = [_i64]
    L.fft_set_default_variant.restype = _int
    L.fft_set_default_variant.argtypes = [_i64, _int]
    L.fft_get_default_variant.restype = _int
    L.fft_get_default_variant.argtypes = [_i64]
    L.fft_variant_dtype.restype = _int
    L.fft_variant_dtype.argtypes = [_i64, _int]
    L.fft_plan_set_wait_limit.restype = _int
    L.fft_plan_set_wait_limit.argtypes = [_vp, ctypes.c_uint64]
    L.fft_plan_create_ragged.restype = _int
    L.fft_plan_create_ragged.argtypes = [ctypes.POINTER(_i64), _i64, _int, _int, _u32, ctypes.POINTER(_vp)]
    L.fft_ragged_variant_count.restype = _int
    L.fft_ragged_variant_count.argtypes = []
    L.fft_set_default_ragged_variant.restype = _int
    L.fft_set_default_ragged_variant.argtypes = [_int]
    L.fft_get_default_ragged_variant.restype = _int
    L.fft_get_default_ragged_variant.argtypes = []
    L.fft_execute_noalloc.restype = _int
    L.fft_execute_noalloc.argtypes = [_i64, _i64, _int, _u32, _vp, _vp, _vp]
    L.fft_twiddle_fp32.restype = None
    L.fft_twiddle_fp32.argtypes = [_i64, _i64, ctypes.POINTER(ctypes.c_float)]
    return L


def check(status: int, what: str = "") -> None:
    if status != 0:
        raise FFTError(status, what)


# --- the C-ABI under its own names -----------------------------------------

def fft_plan_create(n: int, batch: int, direction: int = FFT_FORWARD, dtype: int = FFT_C64) -> int:
    h = _vp()
    check(lib().fft_plan_create(n, batch, direction, dtype, ctypes.byref(h)), "fft_plan_create")
    return h.value


def fft_plan_create_ex(n: int, batch: int, direction: int, dtype: int, flags: int) -> int:
    h = _vp()
    check(lib().fft_plan_create_ex(n, batch, direction, dtype, flags, ctypes.byref(h)),
          "fft_plan_create_ex")
    return h.value


def fft_execute(plan: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    check(lib().fft_execute(plan, in_ptr, out_ptr, stream), "fft_execute")


def fft_plan_get_error(plan: int) -> int:
    return lib().fft_plan_get_error(plan)


def fft_plan_destroy(plan: int) -> None:
    check(lib().fft_plan_destroy(plan), "fft_plan_destroy")


def fft_plan_get_info(plan: int) -> PlanInfo:
    info = PlanInfo()
    check(lib().fft_plan_get_info(plan, ctypes.byref(info)), "fft_plan_get_info")
    return info


def fft_validate(n: int, batch: int, direction: int = 0, dtype: int = 0, flags: int = 0) -> int:
    return lib().fft_validate(n, batch, direction, dtype, flags)


def fft_twiddle_fp32(m: int, k: int) -> complex:
    out = (ctypes.c_float * 2)()
    lib().fft_twiddle_fp32(m, k, out)
    return complex(out[0], out[1])


def fft_variant_count(n: int) -> int:
    return lib().fft_variant_count(n)


def fft_set_default_variant(n: int, variant: int) -> None:
    check(lib().fft_set_default_variant(n, variant), "fft_set_default_variant")


def fft_get_default_variant(n: int) -> int:
    return lib().fft_get_default_variant(n)


def fft_plan_set_wait_limit(plan: int, nanoseconds: int) -> None:
    check(lib().fft_plan_set_wait_limit(plan, nanoseconds), "fft_plan_set_wait_limit")


def fft_execute_noalloc(n: int, batch: int, direction: int, flags: int, in_ptr: int, out_ptr: int,
                        stream: int = 0) -> None:
    """The transform without a plan or any device allocation (static scratch)."""
    check(lib().fft_execute_noalloc(n, batch, direction, flags, in_ptr, out_ptr, stream),
          "fft_execute_noalloc")


def fft_plan_create_ragged(offsets, direction: int = FFT_FORWARD, dtype: int = FFT_C64,
                           flags: int = 0) -> int:
    """offsets: sequence of count+1 int64 element offsets (host)."""
    arr = (ctypes.c_int64 * len(offsets))(*[int(v) for v in offsets])
    h = _vp()
    check(lib().fft_plan_create_ragged(arr, len(offsets) - 1, direction, dtype, flags, ctypes.byref(h)),
          "fft_plan_create_ragged")
    return h.value


def fft_ragged_variant_count() -> int:
    return lib().fft_ragged_variant_count()


def fft_set_default_ragged_variant(variant: int) -> None:
    check(lib().fft_set_default_ragged_variant(variant), "fft_set_default_ragged_variant")


def fft_get_default_ragged_variant() -> int:
    return lib().fft_get_default_ragged_variant()


DTYPE_NAMES = {FFT_C64: "c64", FFT_C64_TC_F16: "tc_f16", FFT_C64_TC_BF16: "tc_bf16", FFT_C32: "c32"}


def fft_variant_dtype(n: int, variant: int) -> int:
    return lib().fft_variant_dtype(n, variant)


def fft_execute_host(plan: int, in_host: int, out_host: int, stream: int = 0) -> None:
    check(lib().fft_execute_host(plan, in_host, out_host, stream), "fft_execute_host")


def fft_execute_c32(plan: int, in_ptr: int, in_exp_ptr: int, out_ptr: int, out_exp_ptr: int,
                    stream: int = 0) -> None:
    check(lib().fft_execute_c32(plan, in_ptr, in_exp_ptr, out_ptr, out_exp_ptr, stream), "fft_execute_c32")
