"""bench.py's reference arm needs no GPU (it times the CPU oracle): its JSON line carries the
contract's keys, its metric and unit match the GPU arm's, under a multi-rank launch only
rank 0 prints, and the process never loads the CUDA library (only the oracle runs there)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# runs the reference arm in-process, then reports on stderr whether the product package was
# imported or its shared library mapped
_PROG = """
import sys
sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"]
import bench
rc = bench.main()
maps = open("/proc/self/maps").read()
sys.stderr.write("PRODUCT_LOADED=%d\\n" % int("paper_1412_0544_gb300" in sys.modules or "librk4chain" in maps))
sys.exit(rc)
"""


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", _PROG], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "PRODUCT_LOADED=0" in r.stderr, r.stderr[-2000:]
    return r.stdout


def test_reference_line():
    out = _run({})
    line = json.loads(out.strip().splitlines()[-1])
    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "site-steps/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.WORKLOAD


def test_reference_other_ranks_are_silent():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}).strip() == ""
