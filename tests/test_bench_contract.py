"""bench.py's host-side pieces (no GPU): the committed ncu traffic record
belongs to the current one-column SpMV source, the roofline peak falls
back when the measured one is absent, and the command-line modes parse."""
import json
import os
import sys

import bench


def test_traffic_record_matches_the_current_kernel_source():
    """The ncu traffic figure in profiles/ is used only while k_spmv1 and its
    launchers hash to the recorded fingerprint: a kernel edit must come with
    a fresh capture (else the bench reports traffic null)."""
    assert bench.recorded_traffic() is not None, bench.kernel_fingerprint()
    assert 1.0e8 < bench.recorded_traffic() < 1.2e8


def test_deblur2048_records_match_the_current_kernel_sources():
    """The ncu DRAM records of the 2048^2 step's banded passes and V-cycle
    are used only while the kernel sources hash to their fingerprints: a
    kernel edit must come with a fresh capture (else traffic is null)."""
    band = bench.recorded_float("k_band", "dram_bytes_per_apply")
    cyc = bench.recorded_float("vcycle", "dram_bytes_per_cycle")
    assert band is not None, bench.source_fingerprint("k_band")
    assert cyc is not None, bench.source_fingerprint("vcycle")
    n = 2048 * 2048
    assert 4 * n * 4 < band < 7 * n * 4   # at least p, u, w_s, w_e once; at most the 7 * 4n of the algorithm
    assert 10 * n < cyc < 100 * n
    levels = bench.recorded("vcycle")
    assert any(k.startswith("level_") for k in levels)


def test_peak_is_measured_or_the_stated_fallback(tmp_path, monkeypatch):
    peak, kind = bench.measured_hbm_peak()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_peak() == (6800.0, "fallback")


def test_command_line_modes_parse(monkeypatch):
    for argv in (["bench.py"], ["bench.py", "--gpus", "2", "--steps", "4", "--warmup", "3"],
                 ["bench.py", "--impl", "reference"], ["bench.py", "--compare-precond"],
                 ["bench.py", "--compare-algorithm2"], ["bench.py", "--profile-iters", "48", "--profile-precond", "2"],
                 ["bench.py", "--no-serve", "--no-cpu", "--no-plain", "--precision", "fp64", "--mode", "batched"],
                 ["bench.py", "--workload", "ct256"], ["bench.py", "--workload", "deblur2048", "--impl", "reference"]):
        monkeypatch.setattr(sys, "argv", argv)
        args = bench.parse()
        assert args.warmup >= 3 or "--warmup" not in argv
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.steps, a.warmup, a.impl, a.workload) == (1, 5, 3, "ours", "deblur2048")
