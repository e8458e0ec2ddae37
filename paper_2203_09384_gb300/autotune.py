"""Autotuner for the schedule variants (tile shape, radix split, prefetch).

For each transform length the library compiles several schedules (see
csrc/schedules.h); for ragged batches it compiles several work-list
kernels (fft_ragged_variant_count).  This module times every candidate on
the device with CUDA events on a synthetic batch of the requested shape,
keeps the fastest, makes it the default through the C-ABI
(fft_set_default_variant) and records the choice in a JSON cache keyed by
GPU name, library version and the compiled variant table, so later processes
start from the tuned table (load_cache) without re-measuring.

Cache location: $GBFFT_TUNE_CACHE, else ~/.cache/gbfft/tune.json.  The
package applies it once per process, before its first plan (autoload), unless
GBFFT_TUNE_CACHE is "off".
"""
from __future__ import annotations

import json
import os
import statistics
import threading

import torch

from . import _abi

LENGTHS = [2 ** k for k in range(1, 12)]


def cache_path() -> str:
    env = os.environ.get("GBFFT_TUNE_CACHE")
    if env and env.lower() != "off":
        return env
    return os.path.join(
        os.path.expanduser("~"), ".cache", "gbfft", "tune.json")


def schedule_fingerprint() -> str:
    """The compiled variant table as seen through the C-ABI (count and dtype of
    every variant per length), so that a cached variant number is applied only
    to the table it was measured on."""
    return ";".join(f"{n}:" + "".join(str(_abi.fft_variant_dtype(n, v)) for v in range(_abi.fft_variant_count(n)))
                    for n in LENGTHS) + f";r{_abi.fft_ragged_variant_count()}"


def _device_key(device=None) -> str:
    name = torch.cuda.get_device_name(device)
    return f"{name}|{_abi.lib().fft_version().decode()}|{schedule_fingerprint()}"


def _time(fn, reps: int, warmup: int = 2) -> float:
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune_lengths(lengths=LENGTHS, elems: int = 2 ** 26, reps: int = 7, apply: bool = True,
                 device=None) -> dict:
    """Time every variant of every length on `elems` complex64 elements
    (uniform [-1, 1]); returns {n: {"best": v, "ms": {v: ms}}}."""
    from . import Plan
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    x = (torch.rand(elems, 2, generator=g, device=dev) * 2 - 1)
    x = torch.view_as_complex(x)
    out = torch.empty_like(x)
    result = {}
    for n in lengths:
        timings = {}
        for v in range(_abi.fft_variant_count(n)):
            if _abi.fft_variant_dtype(n, v) != _abi.FFT_C64:
                continue  # tensor-core variants are chosen by dtype, not tuned against FP32
            p = Plan(n, elems // n, variant=v, device=dev)
            timings[v] = _time(lambda: p.execute(x, out), reps)
            if p.error() != 0:
                timings[v] = float("inf")
            p.close()
        best = min(timings, key=timings.get)
        result[n] = {"best": best, "ms": timings}
        if apply:
            _abi.fft_set_default_variant(n, best)
    return result


def tune_ragged(offsets, x: torch.Tensor, out: torch.Tensor, reps: int = 20, inverse: bool = False) -> dict:
    """Time every ragged work-list variant on this batch (as a CUDA graph
    replay, the way it is meant to run); returns {"best": v, "ms": {v: ms}}."""
    from . import RaggedPlan
    timings = {}
    for v in range(_abi.fft_ragged_variant_count()):
        p = RaggedPlan(offsets, inverse=inverse, variant=v, device=x.device)
        graph = p.capture(x, out)
        timings[v] = _time(graph.replay, reps)
        del graph
        p.close()
    best = min(timings, key=timings.get)
    return {"best": best, "ms": timings}


def save_cache(lengths_result: dict | None = None, ragged_result: dict | None = None, path=None,
               device=None) -> str:
    path = path or cache_path()
    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
    entry = data.setdefault(_device_key(device), {})
    if lengths_result:
        entry["plain"] = {str(n): r["best"] for n, r in lengths_result.items()}
    if ragged_result:
        entry["ragged"] = ragged_result["best"]
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return path


def load_cache(path=None, device=None) -> dict:
    """Apply the cached choices for this GPU, if any: the per-length FP32
    defaults (fft_set_default_variant) and the ragged variant
    (fft_set_default_ragged_variant); returns the cache entry."""
    path = path or cache_path()
    if not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            entry = json.load(f).get(_device_key(device), {})
    except (OSError, ValueError):
        return {}
    for n, v in entry.get("plain", {}).items():
        n, v = int(n), int(v)
        # only FP32 complex64 schedules can be a length's default
        if 0 <= v < _abi.fft_variant_count(n) and _abi.fft_variant_dtype(n, v) == _abi.FFT_C64:
            _abi.fft_set_default_variant(n, v)
    rv = entry.get("ragged")
    if isinstance(rv, int) and 0 <= rv < _abi.fft_ragged_variant_count():
        _abi.fft_set_default_ragged_variant(rv)
    return entry


_autoload_done = False
_autoload_lock = threading.Lock()


def autoload(device=None) -> None:
    """Apply the tuning cache once per process, before the first plan is made
    (Plan and RaggedPlan call this), so that tuning done by an earlier process
    resumes.  GBFFT_TUNE_CACHE=off disables it."""
    global _autoload_done
    if _autoload_done:
        return
    with _autoload_lock:
        if _autoload_done:
            return
        _autoload_done = True
        if os.environ.get("GBFFT_TUNE_CACHE", "").lower() == "off":
            return
        if os.path.exists(cache_path()):
            load_cache(device=device)
