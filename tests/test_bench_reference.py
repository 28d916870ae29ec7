"""The reference arm of bench.py (the CPU oracle on a bounded sample) runs
without a GPU, prints one JSON line in the bench format, and never loads the
CUDA library or its binding."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Runs bench.py in this interpreter, then reports whether the product library
# was mapped into the process or its binding imported.
_DRIVER = """
import json, runpy, sys
sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1", "--oracle-sample", "33x33x17"]
runpy.run_path("bench.py", run_name="__main__")
maps = open("/proc/self/maps").read()
print(json.dumps({"libadr_mapped": "libadr" in maps,
                  "binding_imported": any(m.startswith("paper_1712_06091_gb300.adr") or
                                          m.startswith("paper_1712_06091_gb300._lib") for m in sys.modules)}))
"""


def test_reference_arm_line_without_the_library():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", _DRIVER], capture_output=True, text=True, cwd=ROOT, env=env,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = out.stdout.strip().splitlines()
    line, probe = json.loads(lines[-2]), json.loads(lines[-1])
    assert probe == {"libadr_mapped": False, "binding_imported": False}
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["sample"] == [33, 33, 17]
    assert "257x257x129" in line["metric"]
