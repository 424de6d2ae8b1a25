"""bench.py's reference arm runs the serial oracle on the host (no GPU):
its JSON line carries the keys the benchmark contract names."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                        "--n", "12"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["value"] > 0 and out["higher_is_better"] is True
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == out["value"]
    assert cb["host"]["nproc"] >= 1
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["value"] == out["value"]
    # the reference arm runs the GPU arm's own workload: same config dict
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse(["--n", "12"])
    n_dofs, n_e = 3 * 13 ** 3, 12 ** 3
    assert out["config"] == bench.step_config(args, n_dofs, n_e, n_e * 24 * 24, 9 * 37 ** 3,
                                              out["config"]["n_ca"], 1)
    assert out["config"]["n_ca"] == 2 * (3 * 13 * 37 ** 2 + 1)  # closed form, natural numbering
