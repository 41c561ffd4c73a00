"""bench.py keys the recorded DRAM traffic of the FP64 kernel on a hash of its code: editing
comments or spacing keeps the hash (the compiled kernel is the same), editing code changes it."""
import os

import bench

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1412_0544_gb300", "csrc")


def _read(f):
    with open(os.path.join(CSRC, f)) as fh:
        return fh.read()


def test_code_only_drops_comments_and_spacing():
    src = "int a; // note\n/* block\n comment */  int   b;\n\n"
    assert bench.code_only(src) == "int a; int b;"


def test_hash_ignores_comments_not_code():
    base = bench.kernel_hash(_read)
    commented = bench.kernel_hash(lambda f: _read(f) + "\n// an added remark\n/* and another */\n")
    changed = bench.kernel_hash(lambda f: _read(f).replace("fma(cf.dt6", "fma(cf.h2", 1))
    assert commented == base
    assert changed != base


def test_traffic_table_matches_current_code():
    # recorded counters must describe the kernel as it is: after a code change the entries are
    # re-captured or removed (bench.py then reports traffic null)
    assert all(h == bench.kernel_hash() for h, _ in bench.TRAFFIC)
