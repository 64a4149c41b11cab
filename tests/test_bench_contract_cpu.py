"""The benchmark's reference arm on the CPU: its JSON line carries the keys of
the benchmark contract with the headline's metric and workload, the process
loads neither the package nor its CUDA library (the arm times the oracle
alone), and under a multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402  (no package import at module level)

ARGS = ["--impl", "reference", "--steps", "1", "--warmup", "0"]


def run(code_or_args, env=None, script=False):
    cmd = [sys.executable, "-c", code_or_args] if script else [sys.executable, "bench.py"] + code_or_args
    e = dict(os.environ)
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        e.pop(k, None)
    e.update(env or {})
    return subprocess.run(cmd, cwd=ROOT, env=e, capture_output=True, text=True, timeout=300)


def test_reference_line_has_the_contract_keys():
    p = run(ARGS)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "GB/s" and line["higher_is_better"] is True
    assert line["config"] == bench.headline_config(1)  # the same config as the GPU arm prints
    assert line["steps"] == 1 and line["n_gpus"] == 1 and line["value"] > 0 and line["vs_baseline"] is None
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


@pytest.mark.skipif(not os.path.exists("/proc/self/maps"), reason="needs /proc/self/maps")
def test_reference_arm_loads_no_library():
    code = ("import json, runpy, sys\n"
            f"sys.argv = ['bench.py'] + {ARGS!r}\n"
            "runpy.run_path('bench.py', run_name='__main__')\n"
            "maps = open('/proc/self/maps').read()\n"
            "print(json.dumps({'pkg': any(m.startswith('paper_2209_10643_b300') for m in sys.modules),"
            " 'so': 'libupir' in maps}))\n")
    p = run(code, script=True)
    assert p.returncode == 0, p.stderr[-2000:]
    flags = json.loads(p.stdout.strip().splitlines()[-1])
    assert flags == {"pkg": False, "so": False}


def test_reference_arm_prints_on_rank_zero_only():
    p = run(ARGS, env={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
