"""bench.py's reference arm on the CPU: it times the FP64 oracle on the host
cores (the one place besides the cpu_baseline leg where the benchmark runs
oracle/) and prints one JSON line in the benchmark's contract.  Run here on a
small lattice so that it takes seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--n-side", "8"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, lines
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("snapshot GB/s") and d["unit"] == "GB/s" and d["value"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 1)
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["gpu_launches"] == 0 and d["ms_per_step"] > 0
    assert d["config"]["n_elem"] == 8 ** 3 and d["config"]["lx"] == 8 and d["config"]["n_fields"] == 4
    assert d["config"]["workload"].startswith("SEM snapshot reduction: 8^3 = 512 hex elements")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
