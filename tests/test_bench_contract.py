"""The benchmark's reference arm (the FP64 oracle timed on the host cores)
prints the one JSON line of the benchmark contract, with the metric and
unit of the GPU arm; under a multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small_packed_bed",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_contract_line():
    sys.path.insert(0, ROOT)
    import bench
    lines = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    for k in ("value", "ms_per_step"):
        assert isinstance(d[k], float) and d[k] > 0, k
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith("small_packed_bed") and d["config"]["particles"] == 62_500
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert "small packed bed" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_stored_counters_key_on_code_not_comments(tmp_path):
    """The key under which the benchmark keeps a kernel's measured DRAM
    traffic ignores the comments and spacing of its source files but changes
    with their code (a changed kernel reports no traffic until it is
    captured again)."""
    sys.path.insert(0, ROOT)
    import bench
    a = tmp_path / "a.cu"
    a.write_text("int f(int x) {  // add one\n  return x + 1; /* the sum */ }\n")
    b = tmp_path / "b.cu"
    b.write_text("/* header\n   over two lines */\nint f(int x) {\n    return x + 1;   // plus one\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("int f(int x) { return x + 2; }\n")
    assert bench.file_sha(str(a)) == bench.file_sha(str(b))
    assert bench.file_sha(str(a)) != bench.file_sha(str(c))
    for tr in bench.NCU_TRAFFIC.values():
        assert tr["bytes"] > 0 and all(len(sha) == 16 for sha in tr["files"].values())
