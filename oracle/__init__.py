"""FP64 CPU oracle for the batched 1-D C2C DFT (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from it: the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, FP64); this module compiles it
with gcc into ``oracle/_build/`` and calls it through ctypes.

* ``dft_naive``   - Eq. (dft) / Eq. (idft) of the paper (Sec. 3) summed directly, O(N^2).
* ``fft_radix2``  - the recursive radix-2 decimation in time of Eq. (radix2).
* ``grad_weighted_power`` - gradient of sum |W * DFT(x)|^2 (PyTorch convention).

Arrays are numpy ``complex128`` of shape ``[batch, n]`` (complex64 input is
promoted exactly).  ``inverse=True`` applies Eq. (idft) with its 1/N unless
``normalize=False`` (the unnormalised adjoint).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()


def library_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile oracle.c (optionally with planted mistake ``mutant``)."""
    out = library_path(mutant)
    with _lock:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
            return out
        os.makedirs(_BUILD, exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", f"-DORACLE_MUTANT={int(mutant)}", _SRC,
               "-o", tmp, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


_dp = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64


class Oracle:
    """ctypes wrapper around one build of oracle.c."""

    def __init__(self, mutant: int = 0):
        self.mutant = mutant
        self._lib = ctypes.CDLL(build(mutant))
        lib = self._lib
        lib.oracle_dft_naive.argtypes = [_dp, _dp, _i64, _i64, ctypes.c_int, ctypes.c_int]
        lib.oracle_dft_naive.restype = ctypes.c_int
        lib.oracle_fft_radix2.argtypes = [_dp, _dp, _i64, _i64, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int]
        lib.oracle_fft_radix2.restype = ctypes.c_int
        lib.oracle_grad_weighted_power.argtypes = [_dp, _dp, _dp, _dp, _i64, _i64,
                                                   ctypes.c_int]
        lib.oracle_grad_weighted_power.restype = ctypes.c_int
        lib.oracle_mutant_id.argtypes = []
        lib.oracle_mutant_id.restype = ctypes.c_int
        assert lib.oracle_mutant_id() == mutant

    @staticmethod
    def _prep(x):
        x = np.ascontiguousarray(np.asarray(x), dtype=np.complex128)
        squeeze = x.ndim == 1
        if squeeze:
            x = x[None, :]
        if x.ndim != 2:
            raise ValueError("expected shape [batch, n] or [n]")
        return x, squeeze

    @staticmethod
    def _ptr(a):
        return a.ctypes.data_as(_dp)

    def dft_naive(self, x, inverse: bool = False, normalize: bool = True):
        x, sq = self._prep(x)
        y = np.empty_like(x)
        rc = self._lib.oracle_dft_naive(self._ptr(x), self._ptr(y), x.shape[1], x.shape[0],
                                        int(inverse), int(normalize))
        if rc != 0:
            raise ValueError("oracle_dft_naive rejected its arguments")
        return y[0] if sq else y

    def fft_radix2(self, x, inverse: bool = False, normalize: bool = True,
                   threads: int = 1):
        x, sq = self._prep(x)
        y = np.empty_like(x)
        rc = self._lib.oracle_fft_radix2(self._ptr(x), self._ptr(y), x.shape[1], x.shape[0],
                                         int(inverse), int(normalize), int(threads))
        if rc != 0:
            raise ValueError("oracle_fft_radix2 rejected its arguments (n must be 2^k)")
        return y[0] if sq else y

    def grad_weighted_power(self, x, w, threads: int = 1):
        """Return (grad, loss) for loss = sum |w * DFT(x)|^2."""
        x, sq = self._prep(x)
        w, _ = self._prep(w)
        if w.shape != x.shape:
            raise ValueError("x and w must have the same shape")
        g = np.empty_like(x)
        loss = ctypes.c_double(0.0)
        rc = self._lib.oracle_grad_weighted_power(self._ptr(x), self._ptr(w), self._ptr(g),
                                                  ctypes.byref(loss), x.shape[1], x.shape[0],
                                                  int(threads))
        if rc != 0:
            raise ValueError("oracle_grad_weighted_power rejected its arguments")
        return (g[0] if sq else g), loss.value


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(0)
    return _default


def dft_naive(x, inverse=False, normalize=True):
    return default().dft_naive(x, inverse, normalize)


def fft_radix2(x, inverse=False, normalize=True, threads=1):
    return default().fft_radix2(x, inverse, normalize, threads)


def grad_weighted_power(x, w, threads=1):
    return default().grad_weighted_power(x, w, threads)


def reference(x, inverse=False, normalize=True, threads=1):
    """The oracle's answer for a batch: naive DFT for n <= 64, else radix-2."""
    x = np.asarray(x)
    n = x.shape[-1]
    if n <= 64:
        return dft_naive(x, inverse, normalize)
    return fft_radix2(x, inverse, normalize, threads)


MUTANTS = {
    1: "twiddle of the wrong sign in the radix-2 butterfly",
    2: "inverse loses its 1/N",
    3: "naive DFT phase index shifted by one",
    4: "even and odd halves swapped in the radix-2 split",
    5: "radix-2 twiddle dropped",
    6: "gradient loses the factor 2",
    7: "gradient picks up a stray conjugation",
}
