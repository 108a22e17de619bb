"""The bench's reference arm (the oracle on the host cores) keeps the JSON-line contract;
run at a small size on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--m", "64", "--n", "32"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["metric"] == "SVDs/s" and line["unit"] == "SVDs/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["config"]["m"] == 64 and line["config"]["n"] == 32


def test_traffic_records_match_kernel_form_and_sources(tmp_path, monkeypatch):
    """A DRAM traffic record is used only for its own size and kernel form (CTAs per visit)
    and only while the captured sources are unchanged."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    root = tmp_path
    (root / "profiles").mkdir()
    src = root / "k.cu"
    src.write_text("kernel v1")
    sha = hashlib.sha256(b"kernel v1").hexdigest()
    recs = {"records": [
        {"m": 64, "n": 64, "work_cluster": 8, "sources": ["k.cu"], "sources_sha256": sha,
         "bytes_per_launch": 123.0, "how": "cluster capture"},
        {"m": 64, "n": 64, "work_cluster": 1, "sources": ["k.cu"], "sources_sha256": "0" * 64,
         "bytes_per_launch": 456.0, "how": "stale capture"}]}
    (root / "profiles" / "sweep_fp64_traffic.json").write_text(json.dumps(recs))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_record(64, 64, 8) == (123.0, "cluster capture")
    assert bench.traffic_record(64, 64, 1) == (None, "sources changed since the capture")
    assert bench.traffic_record(64, 64, 4)[0] is None
    src.write_text("kernel v2")
    assert bench.traffic_record(64, 64, 8) == (None, "sources changed since the capture")


def test_tensor_flop_model_of_the_blocked_binary32_stage():
    """Visits per sweep of 64-column blocks (k blocks, k even): (k - 1) k / 2; each counts the
    Gram and the application as three TF32 products of 2 m 128^2 flops."""
    sys.path.insert(0, ROOT)
    import bench
    n = 8192
    k = n // 64
    assert bench.tensor_flops_low(n, n, 1) == (k - 1) * (k // 2) * 6 * 2.0 * n * 128 * 128
    assert bench.tensor_flops_low(130, 130, 2) == 2 * 3 * 2 * 6 * 2.0 * 130 * 128 * 128  # 3 blocks -> 4
