"""The benchmark's host-side contract, on CPU: the reference arm (the FP64 oracle timed on a
bounded sample) prints one JSON line with the keys the contract names, ranks other than 0 print
nothing, and the committed DRAM-traffic records are found only for the workload and sources
they were captured on."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--steps", "2", "--warmup", "0", "--workload", "beams64"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["steps"] == 2 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("IMF beams64") and d["config"]["grid"] == [64, 64, 64]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "beams64"],
             {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_traffic_records_match_workload_and_sources():
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for kernel, by_workload in rec.items():
        for workload, r in by_workload.items():
            b = bench.traffic_record(kernel, workload, r["orientations_per_launch"])
            if b is None:
                continue        # the kernel changed since the capture: the line reports null
            assert b == pytest.approx(r["bytes_per_launch"]), (kernel, workload)
            # scaled by the orientations of a launch
            half = bench.traffic_record(kernel, workload, r["orientations_per_launch"] / 2)
            assert half == pytest.approx(r["bytes_per_launch"] / 2)
    # no record for a workload it was not captured on, nor for an unknown kernel
    assert bench.traffic_record("fft_z_inv_mul", "beams64") is None
    assert bench.traffic_record("no_such_kernel", "beams256") is None


def test_traffic_record_rejects_changed_sources(tmp_path, monkeypatch):
    import bench
    rec = {"k": {"w": {"source_sha256_16": "0" * 16, "sources": ["bench.py"], "workload": "w",
                       "orientations_per_launch": 8, "bytes_per_launch": 100}}}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(rec))
    (tmp_path / "bench.py").write_text("# not the captured source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("k", "w") is None
