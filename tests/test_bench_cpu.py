"""The benchmark's host-side contract, without a GPU: the reference arm (the FP64 oracle on
the host cores) prints one JSON line with the contract's keys; the profile summary is read
only when it was taken on the current kernel sources; workload and kernel names."""
import json
import os
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--edge", "16"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "MLUPS"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == bench.host_cores()
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["box"] == [16, 16, 16] and "workload" in line["config"]


def test_profiled_traffic_requires_the_current_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    assert bench.profiled_traffic("k", 64) is None  # no summary
    f = tmp_path / "k_64cubed.md"
    f.write_text("text\ntraffic_bytes_per_launch: 1234 (sources 0123456789abcdef)\n")
    assert bench.profiled_traffic("k", 64) is None  # other sources
    f.write_text(f"traffic_bytes_per_launch: 1234 (sources {bench.kernel_source_hash()})\n")
    assert bench.profiled_traffic("k", 64) == 1234.0
    # AA summaries are checked against the hash that also covers the AA sources
    g = tmp_path / "step_aa_pair_f16_128_64cubed.md"
    g.write_text(f"traffic_bytes_per_launch: 99 (sources {bench.kernel_source_hash()})\n")
    assert bench.profiled_traffic("step_aa_pair_f16_128", 64) is None
    g.write_text(f"traffic_bytes_per_launch: 99 (sources {bench.kernel_source_hash(bench.AA_KERNEL_SOURCES)})\n")
    assert bench.profiled_traffic("step_aa_pair_f16_128", 64) == 99.0


def test_source_hash_ignores_comments():
    src = 'int a = 1; // one\n/* block\n comment */ const char* s = "//not a comment";\nchar q = \'"\';\n'
    assert bench.strip_comments(src) == 'int a = 1;\n const char* s = "//not a comment";\nchar q = \'"\';'
    assert bench.strip_comments("x = 1;\n\n// gone\ny = 2;") == "x = 1;\ny = 2;"


def test_workload_and_kernel_names():
    args = types.SimpleNamespace(edge=128, tau=0.8, kT=1e-4, storage="f32", init="rest", pattern="pingpong")
    w = bench.workload(args)
    assert w["sites"] == 128 ** 3 and w["streaming"] == "pull, ping-pong" and "2 population buffers" in w["l2"]
    args.pattern, args.storage = "aa", "f16"
    w = bench.workload(args)
    assert w["streaming"] == "AA, one buffer in place" and "1 population buffer" in w["l2"]
    assert bench.kernel_name(2, 128, 1e-4, 0) == ("step_tma<f32, 128, Reg, noise>", "step_tma_f32_128")
    assert bench.kernel_name(2, 64, 0.0, 1, "f16", "aa")[1] == "step_aa_f16_64_kt0_bgk"
    assert bench.kernel_name(1, 0, 1e-4, 0)[0] == "step_pull<f32, Reg, noise>"
    assert bench.kernel_name(2, 128, 1e-4, 0, "f16", "pingpong", 2) == (
        "step_tma_pair<f16, 128, Reg, noise>", "step_tma_pair_f16_128")
    assert bench.kernel_name(2, 128, 0.0, 0, "f16", "aa", 2)[1] == "step_aa_pair_f16_128_kt0"
    assert bench.kernel_name(2, 128, 1e-4, 0, "f32", "aa", 1, 2) == (
        "step_aa_even+step_aa_odd_pair<f32, 128, Reg, noise>", "step_aa_oddpair_f32_128")
    assert len(bench.kernel_source_hash()) == 16


def test_mode_norms_match_the_oracle():
    """The FDT accuracy figure divides each mode variance by rho0 kT b_k / cs2 with the
    benchmark's own norm table; it must be Table II's (the oracle's pinned norms)."""
    import numpy as np
    from oracle import rflbm_oracle as o
    assert np.allclose(bench.mode_norms(), o.norms(), rtol=0, atol=1e-15)
