"""The library's default parameters, the oracle's defaults and the benchmark's paper workload
use the values the paper states (tests/golden/paper_parameters.txt, each with its section)."""
import os

import bench
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_parameters.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                name, value = line.split()[:2]
                vals[name] = float(value)
    return vals


def test_library_defaults_are_the_papers():
    import ctypes
    import paper_1412_0544_gb300 as rk
    g = _golden()
    p = rk.rk4_params()
    rk._lib.rk4_params_default(ctypes.byref(p))
    assert (p.a, p.b, p.c) == (g["a"], g["b"], g["c"])


def test_oracle_defaults_are_the_papers():
    g = _golden()
    a, b, c = oracle.params()[:3]
    assert (a, b, c) == (g["a"], g["b"], g["c"])


def test_bench_paper_workload_is_the_papers():
    g = _golden()
    assert bench.PAPER_N == g["N"] and bench.PAPER_STEPS == g["T"] and bench.DT == g["dt"] and bench.D == g["D"]
