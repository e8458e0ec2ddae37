"""Benchmark: batched FP32 C2C FFT sweep, N = 2^1 .. 2^11, N * batch = 2^28.

One step = one forward transform per length (11 launches), each over 2^28
complex64 elements (2 GiB in, 2 GiB out), re/im iid U[-1, 1] drawn on the
device from seed 1.  Inputs are 16x the L2 size, so no flush is needed.

Metric: HBM GB/s of algorithmic traffic (16 bytes per element: one 8-byte
read, one 8-byte write) over the whole step, summed over ranks.  Also printed:
per-length GB/s and 5 N log2 N GFLOP/s, the roofline of the dominant kernel
against the measured copy bandwidth, the end-to-end rate through the C-ABI
with pinned host buffers, clocks sampled during the timed region, and the FP64
CPU oracle timed on a bounded sample (the CPU baseline).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 launch under torch.distributed.run; every rank transforms its own
2^28-element batches (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LOG2NS = list(range(1, 12))
ELEMS = 2 ** 28                   # complex64 elements per length per rank
BYTES_PER_ELEM = 16               # 8 B read + 8 B write
METRIC = "Batched C2C FFT HBM GB/s (% of peak) N=2..2048; TC-fp16 vs fp32 at fixed err"
WORKLOAD = "fp32 batched C2C forward FFT sweep N=2^1..2^11, N*batch=2^28 complex64, U[-1,1], seed 1"
KERNEL_SOURCES = ["fft_device.cuh", "fft_kernels.cu", "schedules.h"]


def flops_per_elem(n: int) -> float:
    return 5.0 * math.log2(n)


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def strip_comments(src: str) -> str:
    """C/C++/CUDA source without comments and with whitespace runs collapsed
    (string and character literals kept as written), so that an edit to a
    comment leaves the hash of the code unchanged."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
            out.append(" ")
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash() -> str:
    """Hash of the kernel sources' code (comments and layout ignored): the
    stored DRAM traffic is used only while the code it was captured from is
    unchanged."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2203_09384_gb300", "csrc", name), encoding="utf-8") as f:
            h.update(strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(log2n: int, path: str | None = None):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel sources changed since it was captured."""
    p = path or os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash():
        return None
    v = d.get("bytes_per_launch", {}).get(str(2 ** log2n))
    return float(v) if v is not None else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, max clock, throttle reasons seen Active, sample
        count and peak power from nvidia-smi CSV lines (FIELDS order)."""
        sm, smax, power, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def cpu_baseline(budget_s: float = 12.0, threads: int | None = None):
    """The FP64 oracle (recursive radix-2, threaded over signals), as it stands,
    on a bounded sample of the same workload: for every length, the first
    signals of the seed-1 U[-1,1] input, about budget/11 seconds each."""
    import numpy as np
    import oracle
    import synth

    threads = threads or os.cpu_count() or 1
    per_n = budget_s / len(LOG2NS)
    total_bytes, total_t, detail = 0.0, 0.0, {}
    for k in LOG2NS:
        n = 2 ** k
        rows = max(64, 2 ** 14 // n)
        while True:
            x = synth.uniform(rows, n, seed=1).numpy().astype(np.complex128)
            t0 = time.perf_counter()
            oracle.fft_radix2(x, threads=threads)
            dt = time.perf_counter() - t0
            if dt >= per_n / 4 or rows * n >= ELEMS:
                break
            rows = min(ELEMS // n, rows * max(2, int(per_n / 4 / max(dt, 1e-4))))
        # rescale to the time budget
        elems = rows * n
        total_bytes += BYTES_PER_ELEM * elems
        total_t += dt
        detail[str(n)] = round(BYTES_PER_ELEM * elems / dt / 1e9, 4)
    return {"value": round(total_bytes / total_t / 1e9, 4), "unit": "GB/s", "cores": threads,
            "kind": "oracle",
            "sample": f"FP64 recursive radix-2 on the first signals of each length's seed-1 input, "
                      f"{total_bytes / BYTES_PER_ELEM / 1e6:.1f} M elements in {total_t:.1f} s "
                      f"(about {budget_s:.0f} s of CPU work)",
            "per_n_gbs": detail}


def sample_stats(ms: list) -> dict:
    """Mean, median, minimum ("optimal") and standard deviation of per-call or
    per-step times (ms)."""
    return {"mean": round(statistics.mean(ms), 4), "median": round(statistics.median(ms), 4),
            "min": round(min(ms), 4), "std": round(statistics.pstdev(ms), 4)}


def tc_stage_count(info) -> int:
    """Radix-16 stages a plan runs on tensor cores (0 for an FP32 plan)."""
    return int(info.tc_stages)


def _time_ms(fn, stream, reps: int = 10, warmup: int = 3, inner: int = 1) -> float:
    """Median over `reps` samples of the CUDA-event time per call; each sample
    times `inner` calls enqueued back to back (inner = 1: one call's latency,
    including the gap while the host enqueues it; inner > 1: the device's
    throughput for repeated calls, as in the sweep)."""
    import torch
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(inner):
            fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b) / inner)
    return statistics.median(ts)


EXTRAS = ("adjoint", "ragged", "precision")


def run_extras(dev, stream, peak, which=EXTRAS, ragged_variant=None):
    """The other workloads of the hot path, each on its own synthetic data:
    the adjoint (autograd backward), ragged mixed lengths in one graph-captured
    launch, and FP16/BF16 tensor-core radix-16 stages against FP32."""
    out = {}
    if "adjoint" in which:
        out["adjoint"] = extra_adjoint(dev, stream)
    if "ragged" in which:
        out["ragged"] = extra_ragged(dev, stream, ragged_variant)
    if "precision" in which:
        out["precision"] = extra_precision(dev, stream, peak)
    return out


def _gbs(elems, ms):
    return round(BYTES_PER_ELEM * elems / (ms * 1e-3) / 1e9, 1)


def extra_adjoint(dev, stream):
    """loss = sum |W * FFT(x)|^2, N = 1024, batch = 65536, seed 2: forward and
    adjoint (unnormalised inverse) kernels and one autograd step."""
    import torch

    import paper_2203_09384_gb300 as gb

    n, b = 1024, 65536
    g = torch.Generator(device=dev)
    g.manual_seed(2)
    x = torch.view_as_complex(torch.randn(b, n, 2, generator=g, device=dev))
    w = torch.view_as_complex(torch.randn(b, n, 2, generator=g, device=dev))
    fwd = gb.Plan(n, b, device=dev)
    adj = gb.Plan(n, b, inverse=True, normalized=False, device=dev)
    y = torch.empty_like(x)
    ms_f = _time_ms(lambda: fwd.execute(x, y), stream, inner=10)
    ms_b = _time_ms(lambda: adj.execute(y, x), stream, inner=10)
    xg = x.clone().requires_grad_(True)

    def step():
        xg.grad = None
        loss = (torch.abs(w * gb.FFTFunction.apply(xg)) ** 2).sum()
        loss.backward()

    ms_step = _time_ms(step, stream, reps=5)
    return {"workload": "loss=sum|W*FFT(x)|^2, N=1024, batch=65536, x,W ~ CN(0,1), seed 2",
            "forward_gbs": _gbs(n * b, ms_f), "adjoint_backward_gbs": _gbs(n * b, ms_b),
            "forward_ms": round(ms_f, 4), "adjoint_ms": round(ms_b, 4),
            "autograd_step_ms": round(ms_step, 4),
            "timing": "kernels: 10 calls back to back per sample, median of 10 samples",
            "note": "step = forward FFT + torch loss ops + adjoint FFT kernel"}


def extra_ragged(dev, stream, variant=None):
    """20000 signals, lengths 2^U{4..11}, seed 3: one ragged launch replayed
    from a CUDA graph, against one plain launch per length (also a graph) on
    the same signals and a uniform N = 2048 call of the same element count.
    The ragged variant is the tuner's pick unless `variant` names one."""
    import torch

    import paper_2203_09384_gb300 as gb
    import synth
    from paper_2203_09384_gb300 import autotune

    lengths = synth.ragged_lengths(20000, seed=3)
    offs = synth.ragged_offsets(lengths)
    xr = synth.ragged_uniform(lengths, seed=3).to(dev)
    yr = torch.empty_like(xr)
    if variant is None:
        tuned = autotune.tune_ragged(offs.numpy(), xr, yr, reps=10)
    else:
        tuned = {"best": int(variant), "ms": {}}
    rp = gb.RaggedPlan(offs.numpy(), variant=tuned["best"], device=dev)
    total = int(offs[-1])
    # the same signals grouped by length: one plain launch per length
    grouped, pos = [], 0
    for L in sorted(set(lengths.tolist())):
        cnt = int((lengths == L).sum())
        grouped.append((L, cnt, pos))
        pos += L * cnt
    plans = [(gb.Plan(L, cnt, device=dev), p0, L * cnt) for L, cnt, p0 in grouped]
    nu = 2048
    bu = total // nu
    uni = gb.Plan(nu, bu, device=dev)
    # 163 MB of traffic would sit in the 129 MB L2 after one replay: rotate
    # through 8 buffer pairs (1.3 GB) so every replay reads and writes HBM
    rot = 8
    bufs = [(xr.clone(), torch.empty_like(xr)) for _ in range(rot)]

    def capture(fn):
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            fn()
        stream.wait_stream(side)
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            fn()
        return gr

    rg = [capture(lambda a=a, o=o: rp.execute(a, o)) for a, o in bufs]
    pg = [capture(lambda a=a, o=o: [p.execute(a[p0:p0 + m], o[p0:p0 + m]) for p, p0, m in plans])
          for a, o in bufs]
    ug = [capture(lambda a=a, o=o: uni.execute(a[:bu * nu], o[:bu * nu])) for a, o in bufs]
    state = {"i": 0}

    def replay(graphs):
        graphs[state["i"] % rot].replay()
        state["i"] += 1

    ms_r = _time_ms(lambda: replay(rg), stream, reps=40, warmup=rot)
    ms_p = _time_ms(lambda: replay(pg), stream, reps=40, warmup=rot)
    ms_u = _time_ms(lambda: replay(ug), stream, reps=40, warmup=rot)
    # device throughput: the 8 graphs replayed back to back per sample
    bt_r = _time_ms(lambda: replay(rg), stream, reps=10, warmup=rot, inner=rot)
    bt_p = _time_ms(lambda: replay(pg), stream, reps=10, warmup=rot, inner=rot)
    bt_u = _time_ms(lambda: replay(ug), stream, reps=10, warmup=rot, inner=rot)
    return {"workload": "20000 C2C FFTs, lengths 2^U{4..11} (seed 3), packed, U[-1,1]",
            "elements": total, "variant": tuned["best"], "tuner_ms": tuned["ms"],
            "ragged_graph_ms": round(ms_r, 4), "ragged_gbs": _gbs(total, ms_r),
            "plain_per_length_graph_ms": round(ms_p, 4), "plain_per_length_gbs": _gbs(total, ms_p),
            "uniform_same_size_graph_ms": round(ms_u, 4), "uniform_same_size_gbs": _gbs(bu * nu, ms_u),
            "uniform_same_size": f"N={nu} x {bu} (one plain launch)",
            "back_to_back": {"ragged_ms": round(bt_r, 4), "ragged_gbs": _gbs(total, bt_r),
                             "plain_per_length_ms": round(bt_p, 4), "plain_per_length_gbs": _gbs(total, bt_p),
                             "uniform_same_size_ms": round(bt_u, 4), "uniform_same_size_gbs": _gbs(bu * nu, bt_u)},
            "timing": "*_graph_ms: one graph replay per CUDA-event sample (latency, with the host's enqueue gap); "
                      "back_to_back: 8 replays per sample (device throughput)",
            "l2": "8 rotating buffer pairs (1.3 GB) so replays are not served from L2",
            "launches": {"ragged": 1, "plain": len(plans), "uniform": 1}}


def extra_precision(dev, stream, peak):
    """FP16/BF16 tensor-core radix-16 stages and complex32 storage against FP32,
    N in {256, 2048}, batch 2^17, signals scaled by 10^U(-3,3), seed 4."""
    import torch

    import paper_2203_09384_gb300 as gb
    import synth

    prec = {}
    for n in (256, 2048):
        b = 2 ** 17
        xs, _ = synth.scaled_normal(b, n, seed=4, device=dev)
        ref = torch.empty_like(xs)
        res = {}
        for dt in ("c64", "tc_f16", "tc_bf16"):
            p = gb.Plan(n, b, dtype=dt, device=dev)
            o = torch.empty_like(xs)
            ms = _time_ms(lambda: p.execute(xs, o), stream, inner=10)
            if dt == "c64":
                ref.copy_(o)
            d = torch.linalg.vector_norm(o - ref, dim=1) / torch.linalg.vector_norm(ref, dim=1)
            res[dt] = {"gbs": _gbs(n * b, ms), "frac": round(_gbs(n * b, ms) / peak, 4), "ms": round(ms, 4),
                       "gelem_s": round(n * b / ms / 1e6, 2),
                       "max_rel_l2_vs_fp32_path": float(d.max()), "tc_stages": tc_stage_count(p.info())}
        # complex32 storage: 4 B per element each way plus one exponent byte per signal
        hs, he = encode_c32(xs)
        p = gb.Plan(n, b, dtype="c32", device=dev)
        ho, hoe = torch.empty_like(hs), torch.empty_like(he)
        ms = _time_ms(lambda: p.execute_c32(hs, he, ho, hoe), stream, inner=10)
        o = decode_c32(ho, hoe)
        d = torch.linalg.vector_norm(o - ref, dim=1) / torch.linalg.vector_norm(ref, dim=1)
        nbytes = 8 * n * b + 2 * b
        res["c32"] = {"gbs": round(nbytes / ms / 1e6, 1), "frac": round(nbytes / ms / 1e6 / peak, 4),
                      "ms": round(ms, 4), "gelem_s": round(n * b / ms / 1e6, 2),
                      "speedup_vs_c64": round(res["c64"]["ms"] / ms, 3),
                      "max_rel_l2_vs_fp32_path": float(d.max()), "tc_stages": 0}
        prec[str(n)] = res
    return {"workload": "CN(0,1) x 10^U(-3,3) per signal (seed 4), batch 2^17",
            "timing": "10 calls back to back per CUDA-event sample, median of 10 samples",
            "note": "error against the FP64 oracle is in the test suite (bound 5e-3 tensor "
                    "core, 2^-11 + 1e-5 complex32 storage); here: difference from the FP32 "
                    "path on the same GPU; c32 input is the complex64 input rounded to "
                    "complex32 storage, its gbs counts 4+4 B per element + 2 B per signal",
            "by_n": prec}


def encode_c32(x: torch.Tensor):
    """complex64 [batch, n] -> complex32 storage (binary16 pairs, exponent per
    signal putting the largest component in [2^14, 2^15)); input preparation."""
    import torch
    ri = torch.view_as_real(x)
    m = ri.abs().amax(dim=(1, 2)).double()
    e = torch.where(m > 0, torch.frexp(m)[1] - 15, torch.zeros_like(m, dtype=torch.int32))
    h = (ri * torch.pow(2.0, -e.double()).float()[:, None, None]).half()
    return h.reshape(x.shape[0], -1).view(torch.complex32), e.to(torch.int8)


def decode_c32(h: torch.Tensor, e: torch.Tensor) -> torch.Tensor:
    import torch
    ri = h.view(torch.float16).float().reshape(h.shape[0], -1, 2)
    return torch.view_as_complex(ri * torch.pow(2.0, e.double()).float()[:, None, None])


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host cores, on this bench's
    workload, each step a bounded sample."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    budget = 6.0
    for _ in range(args.warmup):
        cpu_baseline(budget_s=budget / 4)
    vals = []
    cb = None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cb = cpu_baseline(budget_s=budget)
        vals.append(cb["value"])
    sample_ms = (time.perf_counter() - t0) * 1e3 / max(args.steps, 1)
    value = statistics.mean(vals)
    cb["value"] = round(value, 4)
    # one full step (every length over ELEMS elements) at the sampled rate, so
    # that value * ms_per_step is the step's bytes on both arms
    full_step_ms = BYTES_PER_ELEM * ELEMS * len(LOG2NS) / (value * 1e9) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(full_step_ms, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (bounded CPU sample per step)", "device": "host cpu",
                       "ms_per_step": "one full step's bytes at the sampled rate",
                       "sample_ms_per_step": round(sample_ms, 1)},
            "cpu_baseline": cb,
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def rank_input(rank: int, elems: int, device="cpu"):
    """The batch one rank transforms: its own seeded U[-1, 1] draw (seed
    1 + rank), so ranks work on different data and exchange none of it (the
    sweep is weak scaling: every rank moves the same bytes)."""
    import synth
    return synth.uniform(1, elems, seed=1 + rank, device=device).reshape(-1)


def reduce_max_over_ranks(ms: float, device=None) -> float:
    """The slowest rank's time (the job is done when every rank is done)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_rank: float, world: int, ms: float) -> float:
    """Aggregate rate: the bytes every rank moved over the slowest rank's time."""
    return bytes_per_rank * world / (ms * 1e-3) / 1e9


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2203_09384_gb300 as gb
    import synth

    rank, world, local = env_rank()
    distributed = "RANK" in os.environ  # launched by torch.distributed.run (any world size)
    if distributed:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    # plans and resident inputs (not timed)
    global ELEMS, LOG2NS
    if args.elems:
        ELEMS = int(args.elems)
    if args.only_n:
        LOG2NS = [int(math.log2(int(v))) for v in args.only_n.split(",")]
    x = rank_input(rank, ELEMS, dev)
    variant = None if args.variant < 0 else args.variant
    plans = {k: gb.Plan(2 ** k, ELEMS // 2 ** k, device=dev, dtype=args.dtype, variant=variant) for k in LOG2NS}
    c32 = args.dtype == "c32"
    if c32:
        # complex32 storage: the same U[-1, 1] values rounded to binary16, input
        # exponents 0 (any exponent is valid input); one exponent byte per signal
        # each way, so a length moves 8 B per element + 2 B per signal
        xh = torch.view_as_real(x).half().reshape(-1).view(torch.complex32)
        outh = torch.empty_like(xh)
        ein = {k: torch.zeros(ELEMS >> k, dtype=torch.int8, device=dev) for k in LOG2NS}
        eout = {k: torch.empty(ELEMS >> k, dtype=torch.int8, device=dev) for k in LOG2NS}
        del x
    else:
        out = torch.empty_like(x)
    len_bytes = {k: (8 * ELEMS + 2 * (ELEMS >> k)) if c32 else BYTES_PER_ELEM * ELEMS for k in LOG2NS}

    def step(events=None):
        for i, k in enumerate(LOG2NS):
            p = plans[k]
            if events is not None:
                events[i][0].record(stream)
            if c32:
                gb.fft_execute_c32(p.handle, xh.data_ptr(), ein[k].data_ptr(), outh.data_ptr(), eout[k].data_ptr(),
                                   stream.cuda_stream)
            else:
                gb.fft_execute(p.handle, x.data_ptr(), out.data_ptr(), stream.cuda_stream)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in LOG2NS]
          for _ in range(args.steps)]
    sampler = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                           if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit()
                           else local)
    if distributed:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        step(ev[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if distributed:
        dist.barrier()
    ms = t_start.elapsed_time(t_end)
    per_launch = {k: [ev[s][i][0].elapsed_time(ev[s][i][1]) for s in range(args.steps)]
                  for i, k in enumerate(LOG2NS)}
    per_step = [ev[s][0][0].elapsed_time(ev[s][-1][1]) for s in range(args.steps)]
    ms = reduce_max_over_ranks(ms, dev)
    # correctness spot check of the timed output (last length) before reporting
    assert all(p.error() == 0 for p in plans.values())

    # end-to-end through the C-ABI with pinned host buffers: fft_execute_host
    # pipelines copy-in / transform / copy-out per chunk over three streams
    e2e = None
    if not args.no_e2e and not c32:  # fft_execute_host is complex64 only
        hx = torch.empty(ELEMS, dtype=torch.complex64, pin_memory=True)
        hx.copy_(x)
        hy = torch.empty_like(hx, pin_memory=True)
        hplans = {k: gb.Plan(2 ** k, ELEMS // 2 ** k, device=dev, host_staging=True) for k in LOG2NS}

        def e2e_step():
            for k in LOG2NS:
                gb.fft_execute_host(hplans[k].handle, hx.data_ptr(), hy.data_ptr(), stream.cuda_stream)

        e2e_step()
        torch.cuda.synchronize()
        # each step timed on its own; the median step is robust to a transient
        # slowdown of the host's memory (the machine's host is shared)
        e_steps = max(1, min(args.steps, 5))
        step_ms = []
        for _ in range(e_steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step()
            b.record(stream)
            torch.cuda.synchronize()
            step_ms.append(a.elapsed_time(b))
        e_ms = reduce_max_over_ranks(statistics.median(step_ms), dev)
        e_bytes = BYTES_PER_ELEM * ELEMS * len(LOG2NS)
        e2e = {"value": round(whole_job_gbs(e_bytes, world, e_ms), 3), "unit": "GB/s",
               "h2d_bytes_per_step": 8 * ELEMS * len(LOG2NS),
               "d2h_bytes_per_step": 8 * ELEMS * len(LOG2NS), "ms_per_step": round(e_ms, 3),
               "steps": e_steps, "step_ms": {"median": round(statistics.median(step_ms), 3),
                                             "mean": round(statistics.mean(step_ms), 3),
                                             "min": round(min(step_ms), 3), "max": round(max(step_ms), 3)},
               "api": "fft_execute_host (pinned host buffers, 3-stream chunk pipeline)"}
        for p in hplans.values():
            p.close()
        del hx, hy

    if rank != 0:
        if distributed:
            dist.destroy_process_group()
        return 0

    step_bytes = sum(len_bytes.values())
    ms_per_step = ms / args.steps
    value = whole_job_gbs(step_bytes, world, ms_per_step)
    peak, peak_src = peaks()
    per_n = {}
    for k in LOG2NS:
        avg = statistics.mean(per_launch[k])
        gbs = len_bytes[k] / (avg * 1e-3) / 1e9
        st = sample_stats(per_launch[k])
        per_n[str(2 ** k)] = {"ms": round(avg, 4), "gbs": round(gbs, 1),
                              "frac": round(gbs / peak, 4),
                              "gflops": round(ELEMS * flops_per_elem(2 ** k) / (avg * 1e-3) / 1e9, 1),
                              "ms_median": st["median"], "ms_min": st["min"], "ms_std": st["std"],
                              "gbs_best": round(len_bytes[k] / (st["min"] * 1e-3) / 1e9, 1)}
    dom = max(LOG2NS, key=lambda k: statistics.mean(per_launch[k]))
    dom_ms = statistics.mean(per_launch[dom])
    achieved = len_bytes[dom] / (dom_ms * 1e-3) / 1e9
    traffic = ncu_traffic(dom) if args.dtype == "c64" else None
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"c64": "f32", "tc_f16": "f16-tensor-core+f32", "tc_bf16": "bf16-tensor-core+f32",
                  "c32": "f16-storage+f32"}[args.dtype],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "lengths": [2 ** k for k in LOG2NS],
                   "elements_per_length": ELEMS, "bytes_per_step_per_gpu": step_bytes,
                   "l2": ("inputs 1 GiB per length (complex32), 8x L2: no flush needed" if c32
                          else "inputs 2 GiB per length, 16x L2: no flush needed"),
                   "parallelism": f"replicas x{world}", "step_ms": sample_stats(per_step),
                   "per_n": per_n},
        "roofline": {"bound": "hbm", "kernel": f"fft N={2 ** dom}", "achieved": round(achieved, 1),
                     "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": traffic, "algorithmic_bytes": len_bytes[dom]},
        "e2e": e2e,
        "gpu_launches": args.steps * len(LOG2NS),
        "clocks": clocks,
    }
    extras = [] if args.no_extras else [e for e in args.extras.split(",") if e]
    if extras:
        line["extra"] = run_extras(dev, stream, peak, extras,
                                   None if args.ragged_variant < 0 else args.ragged_variant)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if distributed:
        dist.destroy_process_group()
    return 0


def _csv_dram_bytes(csv_path: str) -> list:
    """dram__bytes_read.sum + dram__bytes_write.sum of every launch in an ncu
    CSV log, in launch order."""
    import csv

    per_id, order = {}, []
    with open(csv_path) as f:
        rows = [r for r in csv.reader(line for line in f if not line.startswith("=="))]
    hdr = rows[0]
    i_id, i_name, i_val = hdr.index("ID"), hdr.index("Metric Name"), hdr.index("Metric Value")
    i_unit = hdr.index("Metric Unit")
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    for r in rows[1:]:
        if len(r) <= i_val or r[i_name] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        if r[i_id] not in per_id:
            per_id[r[i_id]] = 0.0
            order.append(r[i_id])
        per_id[r[i_id]] += float(r[i_val].replace(",", "")) * scale[r[i_unit]]
    return [per_id[i] for i in order]


def write_traffic(csv_paths: str, elems: int, out_path: str | None = None) -> dict:
    """Write profiles/traffic.json from ncu CSV logs of DRAM bytes
    (dram__bytes_read.sum and dram__bytes_write.sum): either one log per
    length (comma-separated, sweep order, one launch each) or one log of one
    sweep step (a launch per length).  Captured at `elems` elements per
    launch and scaled to the benchmark's 2^28, with the hash of the kernel
    sources it describes."""
    paths = [p for p in csv_paths.split(",") if p]
    launches = []
    for p in paths:
        got = _csv_dram_bytes(p)
        launches.extend(got if len(paths) == 1 else got[:1])
    if len(launches) != len(LOG2NS):
        raise SystemExit(f"expected {len(LOG2NS)} launches, found {len(launches)}")
    factor = ELEMS / elems
    note = "dram__bytes_read.sum + dram__bytes_write.sum of one forward launch per length"
    if len(paths) > 1:
        note += ", each length captured on its own"
    if factor != 1:
        note += f", times {factor:g} (traffic grows in proportion to the elements)"
    out = {"source_hash": kernel_source_hash(), "captured_elements": elems, "scaled_to_elements": ELEMS,
           "note": note, "bytes_per_launch": {str(2 ** k): b * factor for k, b in zip(LOG2NS, launches)}}
    with open(out_path or os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out["bytes_per_launch"]))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint / ragged / tensor-core workloads")
    ap.add_argument("--extras", default=",".join(EXTRAS),
                    help="comma list of the extra workloads to run (adjoint, ragged, precision)")
    ap.add_argument("--only-n", default="", help="comma list of lengths (profiling runs)")
    ap.add_argument("--ragged-variant", type=int, default=-1,
                    help="ragged variant of the ragged extra (profiling runs; default: the tuner's pick)")
    ap.add_argument("--elems", type=int, default=0, help="elements per length (profiling runs)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="schedule variant of the length given by --only-n (profiling runs; default: the length's own)")
    ap.add_argument("--dtype", default="c64", choices=["c64", "tc_f16", "tc_bf16", "c32"],
                    help="arithmetic / storage of the sweep (runs of the tensor-core and complex32 paths)")
    ap.add_argument("--write-traffic", default="", metavar="NCU_CSV[,NCU_CSV...]",
                    help="write profiles/traffic.json from ncu DRAM-bytes CSVs (one per length, or one of a "
                         "whole sweep step; captured with --elems, if given) and exit")
    args = ap.parse_args(argv)
    bad = [e for e in args.extras.split(",") if e and e not in EXTRAS]
    if bad:
        ap.error(f"unknown extras: {bad}")
    if args.variant >= 0 and len([v for v in args.only_n.split(",") if v]) != 1:
        ap.error("--variant needs exactly one length in --only-n")
    if args.write_traffic:
        write_traffic(args.write_traffic, args.elems or ELEMS)
        return 0
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
