"""Host-side logic of bench.py, CPU only: the ncu DRAM-traffic CSV parser and
its source-hash guard, the clock-sample summary, the tensor-core stage count
and the FP64 CPU baseline line."""
import json
import types

import bench


def _ncu_csv(path, per_launch, extra_ids=()):
    """An ncu --csv log: a preamble line, then one row per metric and launch."""
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
           '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')
    rows = ["==PROF== Connected to process 1", hdr]
    for i, (rd_mb, wr_mb) in enumerate(per_launch):
        for name, unit, val in (("dram__bytes_read.sum", "Mbyte", f"{rd_mb:,.3f}"),
                                ("gpu__time_duration.sum", "usecond", "650.0"),
                                ("dram__bytes_write.sum", "Gbyte", f"{wr_mb / 1000:.6f}")):
            rows.append(f'"{33 + i}","1","python","h","k{i}","1","7","(128, 1, 1)","(760, 1, 1)","0","10.3",'
                        f'"Command line profiler metrics","{name}","{unit}","{val}"')
    path.write_text("\n".join(rows) + "\n")


def test_write_traffic_sums_and_scales(tmp_path):
    launches = [(2147.5 + k, 2000.0 + 10 * k) for k in range(len(bench.LOG2NS))]
    csv_path = tmp_path / "t.csv"
    _ncu_csv(csv_path, launches)
    out_path = tmp_path / "traffic.json"
    out = bench.write_traffic(str(csv_path), bench.ELEMS // 8, str(out_path))
    assert out["source_hash"] == bench.kernel_source_hash()
    assert out["captured_elements"] * 8 == out["scaled_to_elements"] == bench.ELEMS
    for k, (rd, wr) in zip(bench.LOG2NS, launches):
        got = out["bytes_per_launch"][str(2 ** k)]
        assert abs(got - 8 * (rd + wr) * 1e6) <= 1e-6 * got  # Mbyte and Gbyte units, times 8
    # the bench reads it back only while the kernel sources hash to the capture
    assert bench.ncu_traffic(11, str(out_path)) == out["bytes_per_launch"]["2048"]
    stale = json.loads(out_path.read_text())
    stale["source_hash"] = "0" * 16
    out_path.write_text(json.dumps(stale))
    assert bench.ncu_traffic(11, str(out_path)) is None


def test_write_traffic_from_one_capture_per_length(tmp_path):
    """One CSV per length (each length captured on its own, one launch each,
    in sweep order): the same sums, in the order of the files."""
    launches = [(100.0 + k, 90.0 + k) for k in range(len(bench.LOG2NS))]
    paths = []
    for k, launch in enumerate(launches):
        p = tmp_path / f"n{k}.csv"
        _ncu_csv(p, [launch])
        paths.append(str(p))
    out = bench.write_traffic(",".join(paths), bench.ELEMS // 8, str(tmp_path / "traffic.json"))
    for k, (rd, wr) in zip(bench.LOG2NS, launches):
        got = out["bytes_per_launch"][str(2 ** k)]
        assert abs(got - 8 * (rd + wr) * 1e6) <= 1e-6 * got
    assert "on its own" in out["note"]


def test_write_traffic_rejects_a_short_capture(tmp_path):
    csv_path = tmp_path / "t.csv"
    _ncu_csv(csv_path, [(1.0, 1.0)] * 3)
    try:
        bench.write_traffic(str(csv_path), bench.ELEMS, str(tmp_path / "x.json"))
    except SystemExit as e:
        assert "expected" in str(e)
    else:
        raise AssertionError("a capture with too few launches must be refused")


def test_clock_summary():
    lines = ["0, 2070, 2070, 600.5, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2060, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 1980, 2070, 1380.2, 0x4, Not Active, Not Active, Not Active, Active",
             "garbage line",
             "0, [N/A], 2070, 10, 0x0, Not Active, Not Active, Not Active, Not Active"]
    c = bench.ClockSampler.summarize(lines)
    assert c["samples"] == 3 and c["sm_mhz"] == 2060 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"] and c["power_w_max"] == 1380.2
    assert bench.ClockSampler.summarize([])["sm_mhz"] is None


def test_tc_stage_count():
    """The bench reports the plan's own count of tensor-core stages (a row may
    run only its last radix-16 stage there)."""
    info = types.SimpleNamespace(tc=1, num_stages=3, radix=[8, 16, 16, 0, 0, 0, 0, 0], tc_stages=1)
    assert bench.tc_stage_count(info) == 1
    info.tc, info.tc_stages = 0, 0
    assert bench.tc_stage_count(info) == 0


def test_cpu_baseline_line_is_bounded_and_complete():
    cb = bench.cpu_baseline(budget_s=0.4, threads=2)
    assert cb["kind"] == "oracle" and cb["unit"] == "GB/s" and cb["cores"] == 2
    assert cb["value"] > 0 and set(cb["per_n_gbs"]) == {str(2 ** k) for k in bench.LOG2NS}
    assert "M elements" in cb["sample"]


def test_reference_line_keys(monkeypatch, capsys):
    """The reference arm's JSON line: the contract keys, a full-step time that
    matches its rate, and a zero-byte e2e."""
    fake = {"value": 8.0, "unit": "GB/s", "cores": 4, "kind": "oracle", "sample": "x", "per_n_gbs": {}}
    monkeypatch.setattr(bench, "cpu_baseline", lambda budget_s=0, threads=None: dict(fake))
    monkeypatch.delenv("RANK", raising=False)
    args = type("A", (), {"steps": 2, "warmup": 3})()
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] == 8.0
    step_bytes = bench.BYTES_PER_ELEM * bench.ELEMS * len(bench.LOG2NS)
    assert abs(line["value"] * 1e9 * line["ms_per_step"] * 1e-3 - step_bytes) / step_bytes < 1e-3
    assert line["e2e"] == {"value": 8.0, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_sample_stats():
    st = bench.sample_stats([2.0, 1.0, 4.0, 3.0])
    assert st == {"mean": 2.5, "median": 2.5, "min": 1.0, "std": round(1.25 ** 0.5, 4)}
    assert bench.sample_stats([0.5]) == {"mean": 0.5, "median": 0.5, "min": 0.5, "std": 0.0}


def test_source_hash_ignores_comments_only():
    code = 'int f(int a) { // twice\n  return 2 * a; /* doubled */ }\nconst char* s = "x // y";\n'
    same = '/* header */\nint f(int a) {\n    return 2 * a;  // edited comment\n}\nconst char* s = "x // y";'
    assert bench.strip_comments(code) == bench.strip_comments(same)
    assert bench.strip_comments(code) != bench.strip_comments(code.replace("2 * a", "3 * a"))
    assert bench.strip_comments(code) != bench.strip_comments(code.replace('"x // y"', '"x // z"'))

