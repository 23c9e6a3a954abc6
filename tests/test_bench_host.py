"""Host-side logic of bench.py (no GPU): both arms name the same workload, and
the multi-stream leg's launch count follows the library's size-class rule."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_multi_stream_launch_count():
    b = _bench()
    # the bench set (8x 640x480, 8x 1280x720, 12x 1920x1088, 4x 3840x2160) in
    # 4-block strips: 2,400 + 7,200 | 24,480 | 32,400 strips, three size classes
    assert b.ms_launches_per_step(142) == 2 * 3 + 2
    assert b.ms_launches_per_step(3142) == 2 * 3 + 2  # staging choices do not change the launches
    assert b.ms_launches_per_step(40) == 4
    assert b.ms_launches_per_step(81) == 4


def test_reference_arm_names_the_same_workload():
    b = _bench()
    env = dict(os.environ, PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"] == b.bench_config(1)
    assert line["metric"] == b.METRIC and line["unit"] == b.UNIT and line["higher_is_better"] is True
    assert line["e2e"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"
