"""The benchmark's use of the committed ncu figures of the fused step kernel (CPU only).

The bench line's roofline `traffic` and its `alu` object come from
profiles/step2d_f32_traffic.json, keyed to a hash of the kernel sources; once the sources change
the figures no longer describe the kernel and the bench must report null instead of stale
numbers.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def committed():
    with open(os.path.join(ROOT, "profiles", "step2d_f32_traffic.json")) as f:
        return json.load(f)


def test_counters_used_while_the_source_matches(monkeypatch):
    d = committed()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda precision=32: d["kernel_source_hash"])
    per_site = d["dram_bytes_per_site"]
    assert 150.0 <= per_site <= 170.0  # one read and one write of the state, plus halo re-reads
    assert bench.recorded_traffic(2048) == per_site * 2048 * 2048
    assert bench.recorded_traffic(4096) == 4 * bench.recorded_traffic(2048)
    alu = bench.alu_roofline(4096 * 4096, 0.86, 152)
    assert alu["cycles_per_site"] == d["fma_pipe_cycles_per_site"]
    assert 0.0 < alu["frac"] < 1.0
    assert "%.0f%% busy" % (100 * d["fma_pipe_busy_frac"]) in bench.counters_note()


def test_stale_counters_are_reported_as_null(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_hash", lambda precision=32: "0" * 16)
    assert bench.recorded_step_counters() is None
    assert bench.recorded_traffic(4096) is None
    alu = bench.alu_roofline(4096 * 4096, 0.86, 152)
    assert alu["achieved"] is None and alu["frac"] is None
    assert "no ncu figure" in bench.counters_note()


def test_source_hash_ignores_comments_only():
    code = "int f(int x) {\n    return x + 1;  // one more\n}\n/* block\n   comment */\n"
    assert bench.strip_comments(code) == bench.strip_comments(code.replace("one more", "plus one"))
    assert bench.strip_comments(code) == bench.strip_comments("// header\n" + code)
    assert bench.strip_comments(code) != bench.strip_comments(code.replace("x + 1", "x + 2"))
