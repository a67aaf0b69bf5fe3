"""Host logic of the benchmark's JSON line, on CPU: the roofline object of
the dominant kernel and the DRAM-traffic lookup keyed by the kernel sources'
hash."""
import json
import os

import pytest

import bench


def test_roofline_takes_the_kernel_with_the_largest_device_time(monkeypatch):
    monkeypatch.setattr(bench, "load_peaks", lambda: (6000.0, "measured"))
    monkeypatch.setattr(bench, "load_traffic", lambda name: 1.5e6 if name == "k_b" else None)
    # {name: (launches, total ms, algorithmic bytes)}
    prof = {"k_a": (10, 1.0, 10 * 2e6), "k_b": (4, 2.0, 4 * 6e6), "k_c": (1, 0.5, 1e6)}
    r = bench.roofline(prof)
    assert r["kernel"] == "k_b" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    # 6 MB per launch in 0.5 ms = 12 GB/s
    assert r["achieved"] == pytest.approx(12.0)
    assert r["peak"] == 6000.0 and r["frac"] == pytest.approx(12.0 / 6000.0, abs=1e-4)
    assert r["traffic"] == 1.5e6 and r["launches"] == 4 and r["avg_us"] == pytest.approx(500.0)
    assert r["share"] == pytest.approx(2.0 / 3.5, abs=1e-4)
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r


def test_traffic_only_for_the_kernel_sources_it_was_measured_on(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({
        "k_zinv_epi": {"dram_bytes_per_launch_full_size": 2.5e7, "source_hash": "abc"},
        "k_zfwd": {"dram_bytes_per_launch_full_size": 1.3e7, "source_hash": "old"}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.load_traffic("k_zinv_epi") == 2.5e7
    assert bench.load_traffic("k_zfwd") is None          # measured on other sources
    assert bench.load_traffic("k_plane") is None         # never measured


def test_peaks_come_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6783.5}))
    assert bench.load_peaks() == (6783.5, "measured")


def test_source_hash_ignores_the_host_only_abi_file(tmp_path, monkeypatch):
    # the hash covers the files that define kernels and launch shapes; an edit
    # of the C-ABI's host checks (api.cu) leaves it, an edit of a kernel does not
    import shutil
    src = os.path.join(bench.ROOT, "paper_2601_23002_gb300", "csrc")
    dst = tmp_path / "paper_2601_23002_gb300" / "csrc"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("__pycache__"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    assert len(h0) == 16
    with open(dst / "api.cu", "a") as f:
        f.write("\n// host-side edit\n")
    assert bench.kernel_source_hash() == h0
    with open(dst / "passes.cuh", "a") as f:
        f.write("\n// kernel-side edit\n")
    assert bench.kernel_source_hash() != h0


def test_clock_summary_reads_median_max_and_active_reasons(tmp_path):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1965, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, [N/A], [N/A], [N/A], 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2040, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2040, 20"]                       # cut off when the sampler stopped
    (tmp_path / "clocks.csv").write_text("\n".join(rows) + "\n")
    s = c.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4


def test_clock_summary_without_samples(tmp_path):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "missing.csv")
    assert c.summary()["reasons"] == ["unsampled"]


def _run_bench(args, env_extra=None):
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py")] + args, cwd=bench.ROOT,
                          env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_complete_line():
    # the oracle on the host cores, one bounded sample per step (on the 32^3
    # fcc cell here, to keep the CPU suite short; the default is the 256^3 cell)
    p = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1", "--cell", "1"])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    d = json.loads(lines[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the same config keys as the CUDA arm's line
    from workloads import config_cell
    assert d["config"] == bench.config_dict(1, 1, config_cell(1))
    assert set(d["config"]) == set(bench.config_dict(1, 1))


def test_reference_arm_runs_on_rank_0_only():
    p = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1", "--cell", "1"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0 and p.stdout.strip() == ""
