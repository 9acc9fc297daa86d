"""Host logic of the measurement script (CPU): the DRAM-traffic record is reported only while
the blind rotation's sources are the ones the counters were taken on, and the reference arm
(the oracle on host cores) prints the contract's JSON line on the GPU arm's workload."""
import json
import os
import shutil
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _copy_tree(tmp_path):
    for rel in ["profiles/traffic.json"] + json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[
            "source_files"]:
        path = rel.partition("#")[0]
        dst = tmp_path / path
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, path), dst)


def test_source_hash_marker_cuts_at_the_marker(tmp_path):
    f = tmp_path / "k.cu"
    f.write_text("kernel A\n// Split section\nkernel B\n")
    whole = bench.kernel_source_sha256([str(f)])
    cut = bench.kernel_source_sha256([str(f) + "#// Split section"])
    assert whole != cut
    f.write_text("kernel A\n// Split section\nkernel B changed\n")
    assert bench.kernel_source_sha256([str(f) + "#// Split section"]) == cut   # after the marker: ignored
    assert bench.kernel_source_sha256([str(f)]) != whole


def test_traffic_is_reported_only_for_unchanged_sources(tmp_path, monkeypatch):
    _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = json.load(open(tmp_path / "profiles" / "traffic.json"))
    small = rec["br_kernel"]["small_case"]
    # Make the record describe the copied sources, then change one line of the kernel region.
    rec["source_sha256"] = bench.kernel_source_sha256(rec["source_files"])
    json.dump(rec, open(tmp_path / "profiles" / "traffic.json", "w"))
    # the capture itself reproduces, and a larger launch adds the per-ciphertext bytes only
    assert abs(bench.br_traffic(small["ciphertexts"]) - small["dram_bytes"]) <= 1
    per_ct = (small["dram_bytes"] - bench.BR_KEY_BYTES) / small["ciphertexts"]
    assert abs(bench.br_traffic(65536) - (bench.BR_KEY_BYTES + 65536 * per_ct)) <= 1
    ntt = tmp_path / "paper_2407_19871_gb300" / "csrc" / "ntt.cuh"
    ntt.write_text(ntt.read_text() + "\n// edited\n")
    assert bench.br_traffic(65536) is None
    os.remove(tmp_path / "profiles" / "traffic.json")
    assert bench.br_traffic(65536) is None


@pytest.mark.slow
def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["metric"] == "gate bootstraps/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["config"] == bench.workload_config(1)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
