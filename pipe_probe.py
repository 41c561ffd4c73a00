"""Builds and runs pipe_probe.cu, the microbenchmark behind the arithmetic peaks that bench.py
quotes its ALU rooflines against (FP64 DFMA / DADD / DMUL, FP32 FMA scalar and packed) and the
copy bandwidth.  ``python pipe_probe.py`` prints one JSON line; it needs a GPU.  It includes the
library's per-site arithmetic header (the RK4 step on register-resident sites), but it is a
measurement aid beside the benchmark, not part of the library."""
from __future__ import annotations

import json
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pipe_probe.cu")
EXE = os.path.join(HERE, "_build", "pipe_probe")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def compile_probe() -> str:
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    deps = (SRC, os.path.join(HERE, "paper_1412_0544_gb300", "csrc", "rk4_device.cuh"))
    if not os.path.exists(EXE) or os.path.getmtime(EXE) < max(os.path.getmtime(f) for f in deps):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-o", EXE, SRC]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {SRC}:\n{r.stdout}\n{r.stderr}")
    return EXE


def run() -> dict:
    r = subprocess.run([compile_probe()], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(f"pipe probe failed ({r.returncode}):\n{r.stdout}\n{r.stderr}")
    return json.loads(r.stdout.strip().splitlines()[-1])


if __name__ == "__main__":
    print(json.dumps(run()))
    sys.exit(0)
