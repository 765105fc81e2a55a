"""The benchmark's reference arm on the host: the FP64 oracle timed on a bounded sample of
the MeerKAT-shaped workload (1 h variant, one step of 8 pixels per method).  Checks the
JSON line's contract: metric, unit and direction as the GPU arm, the same config object
(both arms build it with bench.step_config), and the cpu_baseline / e2e objects the
reference arm must carry."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(600)
def test_reference_arm_json_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--workload", "c2_1h"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "smeared-PSF px.vis terms/sec (exact + uv + img)"
    assert line["unit"] == "terms/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "terms/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    import obsgen
    args = argparse.Namespace(workload="c2_1h", prec="tc_fp16")
    K = obsgen.config2_obs(hours=1.0).nvis()
    assert line["config"] == json.loads(json.dumps(bench.step_config(args, K, 128)))
