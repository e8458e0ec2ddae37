"""In-tree build of libgbfft.so for sm_103a (nvcc, no cmake).

The kernels are compiled once per transform length (``-DGBFFT_LOG2N=k``) in
parallel, then linked with the host plan code into one shared library with
the CUDA runtime linked statically.  Outputs go to ``_build/`` beside this
file (git-ignored).  ``python -m paper_2203_09384_gb300.build`` runs it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
# GBFFT_DEBUG build (device-side bounds checks, NaN-poisoned exchanges): a
# separate library for tests, never the one the package loads
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB = os.path.join(BUILD, "libgbfft.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
          "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
LOG2NS = range(1, 12)


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand) and shutil.which(cand) is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbfft.so")
    return cand


def _sources(csrc=CSRC):
    deps = [os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(INCLUDE, "gbfft.h"))
    units = [(os.path.join(csrc, "fft_kernels.cu"), f"fft_kernels_{k}.o", [f"-DGBFFT_LOG2N={k}"])
             for k in LOG2NS]
    units.append((os.path.join(csrc, "gbfft_host.cu"), "gbfft_host.o", []))
    units.append((os.path.join(csrc, "fft_noalloc.cu"), "fft_noalloc.o", []))
    units.append((os.path.join(csrc, "fft_ragged.cu"), "fft_ragged.o", []))
    return units, deps


def _stale(target, inputs):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(i) > t for i in inputs)


def _compile(src, obj, defs, deps, verbose, build_dir=BUILD, extra=()):
    out = os.path.join(build_dir, "obj", obj)
    if not _stale(out, [src] + deps):
        return out, False
    cmd = [nvcc(), *ARCH, *CFLAGS, *extra, "-I", os.path.dirname(src), *defs, "-c", src, "-o", out + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)} {' '.join(defs)}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(out + ".tmp", out)
    return out, True


def build(jobs: int | None = None, verbose: bool = False, force: bool = False,
          csrc: str = CSRC, build_dir: str | None = None, debug: bool = False) -> str:
    """Compile every kernel unit of ``csrc`` and link ``<build_dir>/libgbfft.so``
    (defaults: this package's sources into ``_build/``, or with ``debug`` the
    GBFFT_DEBUG build into ``_build_debug/``); returns its path."""
    build_dir = build_dir or (BUILD_DEBUG if debug else BUILD)
    extra = ("-DGBFFT_DEBUG",) if debug else ()
    lib_path = os.path.join(build_dir, "libgbfft.so")
    os.makedirs(os.path.join(build_dir, "obj"), exist_ok=True)
    units, deps = _sources(csrc)
    if force:
        for _, obj, _ in units:
            p = os.path.join(build_dir, "obj", obj)
            if os.path.exists(p):
                os.remove(p)
    jobs = jobs or min(len(units), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(lambda u: _compile(u[0], u[1], u[2], deps, verbose, build_dir, extra), units))
    objs = [r[0] for r in results]
    if any(r[1] for r in results) or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="--force" in sys.argv, debug="--debug" in sys.argv))
