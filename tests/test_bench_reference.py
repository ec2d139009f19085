"""The reference arm of bench.py (the oracle on this host's cores) prints one JSON line
with the contract's keys, on the CPU, with no GPU involved."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                          "--cpu-procs", "2"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "Gpts/s"
    assert d["config"]["N"] == d["config"]["M"] == 1 << 20 and d["config"]["K"] == 12
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun with N > 1 only rank 0 runs the oracle and prints."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT="29555")
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    assert not [ln for ln in res.stdout.splitlines() if ln.startswith("{")]


def test_committed_traffic_follows_the_kernel_sources(monkeypatch):
    """roofline.traffic is read from the committed in-step capture only while the kernel
    sources hash as they did when it was taken; the figure is the pass's in-step DRAM bytes
    per launch, a whole number of bytes, and unknown kernels give None."""
    sys.path.insert(0, ROOT)
    import bench
    path = os.path.join(ROOT, "profiles", "ncu_step_kernels_n2e20.md")
    txt = open(path).read()
    recorded = txt.split("source_hash:")[1].split()[0]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: recorded)
    for k in ("pass1", "pass2", "passA", "passB"):
        t = bench.committed_traffic(k)
        assert t is not None and t == int(t) and 1e6 < t < 1e9, (k, t)
    row = [ln for ln in txt.splitlines() if ln.startswith("| passA |")][0].split("|")
    assert bench.committed_traffic("passA") == int(row[4])
    assert bench.committed_traffic("nonexistent") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.committed_traffic("passA") is None
