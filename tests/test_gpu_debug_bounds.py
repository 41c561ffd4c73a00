"""The sanitizer substitute: librk4chain_debug.so (built with -DRK4_DEBUG_BOUNDS) checks every
global memory range its kernels read or write and latches RK4_EBOUNDS instead of making an
out-of-range access.  Every case of bounds_cases.py (all schemes, ragged sizes, both
precisions, reductions, sub-domains) must run through it with no check firing (status OK) and
give the release library's bits."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np, torch
import paper_1412_0544_gb300 as rk
import bounds_cases
assert rk.LIB_PATH.endswith("librk4chain_debug.so"), rk.LIB_PATH
ref = np.load(sys.argv[2])
res = bounds_cases.run_all(rk, torch)
report = {}
for name, (arrays, code) in res.items():
    same = all(np.array_equal(np.asarray(a).view(np.uint8), ref[f"{name}__{i}"].view(np.uint8))
               for i, a in enumerate(arrays))
    report[name] = {"status": int(code), "bit_identical": bool(same)}
print(json.dumps(report))
"""


def _load_build():
    import importlib.util
    spec = importlib.util.spec_from_file_location("rk4_build", os.path.join(ROOT, "paper_1412_0544_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_debug_bounds_build_clean_and_bit_identical(tmp_path):
    import torch
    import paper_1412_0544_gb300 as rk
    import bounds_cases
    assert torch.cuda.is_available()
    debug_lib = _load_build().build(debug_bounds=True)
    res = bounds_cases.run_all(rk, torch)
    arrays = {}
    for name, (arrs, code) in res.items():
        assert code == rk.RK4_OK, (name, code)
        for i, a in enumerate(arrs):
            arrays[f"{name}__{i}"] = np.ascontiguousarray(np.asarray(a))
    ref = tmp_path / "ref.npz"
    np.savez(ref, **arrays)
    script = tmp_path / "child.py"
    script.write_text(_CHILD)
    env = dict(os.environ, RK4CHAIN_LIBRARY=debug_lib)
    r = subprocess.run([sys.executable, str(script), ROOT, str(ref)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    report = json.loads(r.stdout.strip().splitlines()[-1])
    assert set(report) == set(res)
    fired = {k: v["status"] for k, v in report.items() if v["status"] != rk.RK4_OK}
    assert not fired, fired
    differ = [k for k, v in report.items() if not v["bit_identical"]]
    assert not differ, differ
