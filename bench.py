"""Benchmark: site-steps/s of classical RK4 on the paper's coupled Roessler chain on GB300.

Workload (one "step" of this benchmark = one pass of the whole hot path): a fixed-end Roessler
chain (Eqs. (6)-(7), a = 0.2, b = 1, c = 9, kappa = 1) of N = 2^27 sites in FP64 (3.2 GB of
state), i.i.d. uniform[-1, 1) initial state from the counter-based generator, advanced 200 RK4
steps with dt = 0.01 by the temporally blocked kernel (tiling chosen by the autotuner),
followed by one FP64 norm reduction with non-finite check.  This is the largest single-GPU
chain configuration; the state and its ping-pong copy are far larger than the 129 MB L2, so no
flush is needed between steps.

Printed: one JSON line (rank 0).  `value` = site-steps/s over all ranks; `roofline` refers to
the blocked FP64 kernel, which is bound by the FP64 pipe (49 FP64 instructions per site-step
against the measured FP64 FMA rate of this GPU); `e2e` measures the same through
rk4_chain_integrate_host from pinned host memory; `cpu_baseline` is the serial C oracle on the
host.  Extra keys report the periodic N = 2^24 chain, the FP32-Kahan path, batches of uneven
chains and the widened schemes.

`--impl reference` times the CPU oracle instead (the reference arm), on bounded samples.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "site-steps/s (RK4, fp64 & fp32-compensated) and % of GB300 HBM roofline"
WORKLOAD = "roessler_chain_fp64_fixed_N2^27_200steps"
N_HEAD, NSTEPS_HEAD, BC_HEAD = 1 << 27, 200, "fixed"  # the timed workload
N_SITES = 1 << 24  # the periodic chain of the extra measurements and the sweeps
NSTEPS = 1000
DT = 0.01
SEED = 0x14120544
D = 3
HBM_GBS_FALLBACK = 6800.0
# Arithmetic peaks for the ALU rooflines, measured by pipe_probe.cu beside this file (run
# by bench.py itself on rank 0 before the workload, so the denominator comes from the same GPU
# and clocks; the constants below, from an earlier probe run on a GB300 at 2070 MHz, are the
# fallback when the probe cannot run).  The classical RK4 Roessler step issues 49 DFMA per
# site-step in FP64 (4 x 7 slope, whose two additions are issued as exact FMAs a*1+b, 9 stage
# states, 12 update), so the roof is the DFMA rate.  FP32: the larger of the scalar and packed
# (f32x2) FMA lane rates.
FP64_INST_PEAK = 0.6272e12
FP32_INST_PEAK = 40.12e12
PEAK_SOURCE = "fallback constants from an earlier pipe_probe run"
PROBE = {}  # the pipe probe's full result in this run (empty without it)


def probe_peaks():
    """Measure the DFMA and FP32 FMA rates with the pipe probe; keep the constants on failure."""
    global FP64_INST_PEAK, FP32_INST_PEAK, PEAK_SOURCE, PROBE
    try:
        import pipe_probe
        r = pipe_probe.run()
        PROBE = r
        FP64_INST_PEAK = float(r["dfma_per_s"])
        FP32_INST_PEAK = float(max(r["ffma_scalar_16chains_per_s"], r["ffma_packed_16lanes_per_s"]))
        PEAK_SOURCE = "of measured: pipe_probe in this run"
        return r
    except Exception as e:  # the probe is a measurement aid; the bench still runs without it
        return {"error": str(e)[:200]}


FP64_INST_PER_SITE_STEP = 49     # DFMA (the slope's 8 additions issued as a * 1 + b)
FP32K_INST_PER_SITE_STEP = 58    # the update: 4 operations per component instead of 1 FMA
# DRAM traffic (read + write bytes) per launch of the FP64 blocked kernel from one ncu capture,
# with the chain length it was taken at: valid only for the kernel code (kernel_hash) and the
# tiling recorded with it; any other combination reports null.  A launch's traffic is
# proportional to the sites it advances (one read and one write of each tile), so a capture at
# N = 2^24 scales to the N = 2^27 workload by the site count.
TRAFFIC = {
    ("24e57e0265074389", "256,4,1"): (402771968 + 357428224, 1 << 24),
    ("24e57e0265074389", "128,4,1"): (402821632 + 356577792, 1 << 24),
    ("24e57e0265074389", "512,2,1"): (402830848 + 356819456, 1 << 24),
    ("24e57e0265074389", "128,8,1"): (403226624 + 356647424, 1 << 24),
    ("24e57e0265074389", "256,4,2"): (402761472 + 357003008, 1 << 24),
    ("24e57e0265074389", "128,4,2"): (402859776 + 356683008, 1 << 24),
    ("24e57e0265074389", "512,2,2"): (402838272 + 357778944, 1 << 24),
    ("24e57e0265074389", "128,8,2"): (402945792 + 357322496, 1 << 24),
    ("24e57e0265074389", "256,8,2"): (402975232 + 357140224, 1 << 24),
}


def traffic_per_launch(khash: str, tiling: dict, n: int):
    """ncu DRAM bytes per launch for this kernel code and tiling, scaled to n sites, or None."""
    rec = TRAFFIC.get((khash, f"{tiling['block']},{tiling['v']},{tiling['k']}"))
    return None if rec is None else rec[0] * n / rec[1]


def code_only(src: str) -> str:
    """C/C++/CUDA source without its comments and blank space, so that an edit of the comments
    alone leaves a kernel's hash (and the counters recorded for it) valid."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


BLOCKED_SOURCES = ("rk4_device.cuh", "rk4_tile.cuh", "k_blocked.cu")
GENERIC_SOURCES = ("rk4_device.cuh", "rk4_tile.cuh", "rk4_generic.cuh", "k_generic.cu")


def kernel_hash(read=None, files=BLOCKED_SOURCES) -> str:
    """Hash of the code (comments and spacing excluded) a kernel is built from: by default the
    blocked kernel; GENERIC_SOURCES for the generic scheme's kernel."""
    read = read or (lambda f: open(os.path.join(ROOT, "paper_1412_0544_gb300", "csrc", f)).read())
    h = hashlib.sha256()
    for f in files:
        h.update(code_only(read(f)).encode())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                mhz.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def host_info() -> dict:
    """The host the CPU baselines ran on: logical core count, architecture, CPU model."""
    import platform
    import subprocess
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu_model": model}


def cpu_baseline(sample_sites: int = 1 << 24, sample_steps: int = 20) -> dict:
    """The serial C oracle on the host (1 core) on a bounded sample of the workload: a
    fixed-end chain made of the workload's first 2^24 sites (the same per-site work), 20 RK4
    steps (about 15 s on one Grace core)."""
    import chain_inputs as ci
    import oracle
    y0 = ci.uniform_state(sample_sites, D, seed=SEED)
    oracle.load()
    t0 = time.perf_counter()
    oracle.rk4_integrate(y0, oracle.ROESSLER, oracle.FIXED, DT, sample_steps)
    dt = time.perf_counter() - t0
    return {"value": sample_sites * sample_steps / dt, "unit": "site-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"fixed-end Roessler chain of the workload's first {sample_sites} sites, {sample_steps} "
                      "RK4 steps, FP64, serial C oracle"}


def run_reference(args):
    """Reference arm: the CPU oracle, timed on bounded samples of the same workload.  Only the
    oracle runs here: the rank comes from the launcher's environment, and the CUDA library is
    never loaded into this process."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import chain_inputs as ci
    import oracle
    oracle.load()
    sites, steps = 1 << 24, 2  # the workload's first 2^24 sites as a fixed-end chain, 2 RK4 steps per step
    y = ci.uniform_state(sites, D, seed=SEED)
    for _ in range(args.warmup):
        y = oracle.rk4_integrate(y, oracle.ROESSLER, oracle.FIXED, DT, steps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y = oracle.rk4_integrate(y, oracle.ROESSLER, oracle.FIXED, DT, steps)
    el = time.perf_counter() - t0
    value = sites * steps * args.steps / el
    sample = (f"fixed-end Roessler chain of the workload's first {sites} sites, {steps} RK4 steps per step, "
              "FP64, serial C oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "site-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sites": N_HEAD, "rk4_steps_per_step": NSTEPS_HEAD, "dt": DT,
                       "boundary": BC_HEAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "site-steps/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "site-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def time_integrate(rk, h, st, cp, ws, nsteps, reps, torch):
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def fp32_kahan_extra(rk, torch, stream, n=1 << 27, nsteps=NSTEPS):
    """FP32 state + Kahan-compensated update on a periodic Roessler chain of N = 2^27 sites,
    1000 steps; its half squared norm against the FP64 GPU path at the same size and steps,
    and its error against the FP64 oracle on a separate 2^16-site chain from the same seed."""
    import chain_inputs as ci
    import oracle
    out = {}
    h = rk.rk4_chain_create(rk.RK4_ROESSLER, rk.RK4_FP32_KAHAN, n, DT, rk.RK4_PERIODIC, None, stream)
    try:
        st = torch.empty((n, D), dtype=torch.float32, device="cuda")
        rk.rk4_fill_uniform(st, n * D, SEED, 0, rk.RK4_FP32_KAHAN, stream)
        cp = torch.zeros_like(st)
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        best = rk.rk4_chain_autotune(h, st.clone(), cp.clone(), ws, 32)
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)  # warm-up: the timed call replays a cached graph
        rk.rk4_fill_uniform(st, n * D, SEED, 0, rk.RK4_FP32_KAHAN, stream)
        cp.zero_()
        e32_0 = rk.rk4_chain_energy(h, st, cp, ws)[0]
        el = time_integrate(rk, h, st, cp, ws, nsteps, 1, torch)
        e32 = rk.rk4_chain_energy(h, st, cp, ws)[0]
        sps = n * nsteps / el
        launches = -(-nsteps // best["k"])
        out.update({"value": sps, "unit": "site-steps/s", "N": n, "steps": nsteps, "tiling": best,
                    "effective_state_GBs": sps * 2 * D * 4 / 1e9,
                    "hbm_traffic_GBs_est": sps * 4 * D * 4 * (1 + 8 * best["k"] / best["G"]) / best["k"] / 1e9,
                    "fp32_pipe_frac_of_measured": sps * FP32K_INST_PER_SITE_STEP / FP32_INST_PEAK,
                    "ms_per_launch": 1e3 * el / launches, "half_norm2_t0": e32_0, "half_norm2_fp32": e32})
        if "rk4_fp32k_regs_lane_ops_per_s" in PROBE:
            # against the same packed instruction stream on register-resident sites (4 sites per
            # thread; with 8, twice the independent work per thread)
            out["frac_of_arithmetic_only"] = sps * FP32K_INST_PER_SITE_STEP / PROBE["rk4_fp32k_regs_lane_ops_per_s"]
            if "rk4_fp32k_regs_v8_lane_ops_per_s" in PROBE:
                out["frac_of_arithmetic_only_v8"] = (sps * FP32K_INST_PER_SITE_STEP /
                                                     PROBE["rk4_fp32k_regs_v8_lane_ops_per_s"])
        del st, cp, ws
    finally:
        rk.rk4_chain_destroy(h)
    # the FP64 GPU path on the same chain, for the norm comparison
    h = rk.rk4_chain_create(rk.RK4_ROESSLER, rk.RK4_FP64, n, DT, rk.RK4_PERIODIC, None, stream)
    try:
        s32 = torch.empty((n, D), dtype=torch.float32, device="cuda")
        rk.rk4_fill_uniform(s32, n * D, SEED, 0, rk.RK4_FP32_KAHAN, stream)
        st64 = s32.double()  # the FP32 start values, widened
        del s32
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_set_tiling(h, 256, 4, 2)
        rk.rk4_chain_integrate(h, st64, None, ws, nsteps)
        e64 = rk.rk4_chain_energy(h, st64, None, ws)[0]
        out["half_norm2_fp64_gpu"] = e64
        out["half_norm2_rel_diff_vs_fp64_gpu"] = abs(out["half_norm2_fp32"] - e64) / abs(e64)
        del st64, ws
    finally:
        rk.rk4_chain_destroy(h)
    # error against the oracle on a separate 2^16-site chain (same seed, FP32 start values)
    m = 1 << 16
    y0 = ci.uniform_state(m, D, seed=SEED).astype(np.float32)
    h = rk.rk4_chain_create(rk.RK4_ROESSLER, rk.RK4_FP32_KAHAN, m, DT, rk.RK4_PERIODIC, None, stream)
    try:
        st = torch.from_numpy(y0).cuda()
        cp = torch.zeros_like(st)
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_set_tiling(h, best["block"], best["v"], best["k"])
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
        got = (st.double() - cp.double()).cpu().numpy()
    finally:
        rk.rk4_chain_destroy(h)
    ref = oracle.rk4_integrate(y0.astype(np.float64), oracle.ROESSLER, oracle.PERIODIC, DT, nsteps)
    out["rel_err_vs_fp64_oracle_2e16"] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    return out


def periodic_fp64_extra(rk, torch, stream, n=N_SITES, nsteps=NSTEPS):
    """The periodic FP64 chain of N = 2^24 sites, 1000 steps, autotuned blocked kernel."""
    h = rk.rk4_chain_create(rk.RK4_ROESSLER, rk.RK4_FP64, n, DT, rk.RK4_PERIODIC, None, stream)
    try:
        st = torch.empty((n, D), dtype=torch.float64, device="cuda")
        rk.rk4_fill_uniform(st, n * D, SEED, 0, rk.RK4_FP64, stream)
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        tiling = rk.rk4_chain_autotune(h, st.clone(), None, ws, 16)
        rk.rk4_chain_integrate(h, st, None, ws, nsteps)  # warm-up with the timed step count (graph cached)
        el = time_integrate(rk, h, st, None, ws, nsteps, 1, torch)
        sps = n * nsteps / el
        return {"value": sps, "unit": "site-steps/s", "N": n, "steps": nsteps, "boundary": "periodic",
                "tiling": tiling, "effective_state_GBs": sps * 2 * D * 8 / 1e9,
                "fp64_pipe_frac_of_measured": sps * FP64_INST_PER_SITE_STEP / FP64_INST_PEAK}
    finally:
        rk.rk4_chain_destroy(h)


def batch_extra(rk, torch, stream, precision, nsteps=NSTEPS):
    """4096 chains, lengths log-uniform in [64, 65536], kappa ~ U[0.5, 2], mixed boundaries:
    the persistent cooperative launch (CUDA graph) and the autotuner's choice between it and
    one blocked launch per k steps, beside one long chain at the same tiling."""
    import chain_inputs as ci
    lengths, kappa, bcs = ci.batch_spec(4096, seed=SEED)
    total = int(lengths.sum())
    h = rk.rk4_batch_create(rk.RK4_ROESSLER, precision, lengths, kappa, bcs, DT, None, stream)
    try:
        dt_ = torch.float32 if precision == rk.RK4_FP32_KAHAN else torch.float64
        st = torch.empty((total, D), dtype=dt_, device="cuda")
        rk.rk4_fill_uniform(st, total * D, SEED, 0, precision, stream)
        cp = torch.zeros_like(st) if precision == rk.RK4_FP32_KAHAN else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        out = {"unit": "site-steps/s", "chains": 4096, "sites": total, "steps": nsteps}
        # the persistent scheme (one cooperative launch, CUDA graph), then the autotuner's choice
        rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_PERSISTENT)
        tp = rk.rk4_chain_autotune(h, st.clone(), cp.clone() if cp is not None else None, ws, 32)
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)  # capture + warm-up
        el = time_integrate(rk, h, st, cp, ws, nsteps, 1, torch)
        out["persistent"] = {"value": total * nsteps / el, "tiling": tp,
                             "kernel": "persistent cooperative, one launch per call, CUDA graph"}
        rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_AUTO)
        best = rk.rk4_chain_autotune(h, st.clone(), cp.clone() if cp is not None else None, ws, 32)
        kern = rk.rk4_chain_get_kernel(h)
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
        el = time_integrate(rk, h, st, cp, ws, nsteps, 1, torch)
        out.update({"value": total * nsteps / el, "tiling": best,
                    "kernel": ("persistent cooperative" if kern == rk.RK4_KERNEL_PERSISTENT
                               else "blocked, one launch per k steps") + ", CUDA graph (autotuned)"})
        del st, cp, ws
    finally:
        rk.rk4_chain_destroy(h)
    # one periodic chain of 2^24 sites with the same tiling and steps: the batch's rate against it
    # measures what uneven chains cost (halos of every chain's last piece, packing, chain lookup)
    n = N_SITES
    h = rk.rk4_chain_create(rk.RK4_ROESSLER, precision, n, DT, rk.RK4_PERIODIC, None, stream)
    try:
        dt_ = torch.float32 if precision == rk.RK4_FP32_KAHAN else torch.float64
        st = torch.empty((n, D), dtype=dt_, device="cuda")
        rk.rk4_fill_uniform(st, n * D, SEED, 0, precision, stream)
        cp = torch.zeros_like(st) if precision == rk.RK4_FP32_KAHAN else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_set_tiling(h, best["block"], best["v"], best["k"])
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
        el = time_integrate(rk, h, st, cp, ws, nsteps, 1, torch)
        out["single_chain_2e24_same_tiling"] = n * nsteps / el
        out["ratio_to_single_chain"] = out["value"] / out["single_chain_2e24_same_tiling"]
        del st, cp, ws
    finally:
        rk.rk4_chain_destroy(h)
    return out


def size_sweep(args):
    """Site-steps/s against chain length N = 2^10 .. 2^27 (the GPU counterpart of the paper's
    size-dependence study, Sec. 3.2.3): the standard scheme (one launch per stage, Sec. 2.2)
    against temporal blocking and the persistent kernel, FP64 and FP32-Kahan, periodic
    Roessler chain.  Prints one JSON object per (N, precision, scheme)."""
    import torch
    import paper_1412_0544_gb300 as rk
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    # "autotuned": RK4_KERNEL_AUTO with a workspace large enough for the staged scheme too, so
    # that rk4_chain_autotune picks the faster of the tiled and the standard scheme
    schemes = [("standard", rk.RK4_KERNEL_STAGED), ("blocked", rk.RK4_KERNEL_BLOCKED),
               ("persistent", rk.RK4_KERNEL_PERSISTENT), ("autotuned", rk.RK4_KERNEL_AUTO)]
    lo, hi = args.sweep_min, args.sweep_max
    tuned = {}  # the paper finds the optimal cluster size independent of N: tune up to 2^22, then reuse
    for p in range(lo, hi + 1):
        n = 1 << p
        for prec, pname in ((rk.RK4_FP64, "fp64"), (rk.RK4_FP32_KAHAN, "fp32_kahan")):
            dtype = torch.float64 if prec == rk.RK4_FP64 else torch.float32
            st0 = torch.empty((n, D), dtype=dtype, device="cuda")
            rk.rk4_fill_uniform(st0, n * D, SEED, 0, prec, stream)
            for sname, kern in schemes:
                h = rk.rk4_chain_create(rk.RK4_ROESSLER, prec, n, DT, rk.RK4_PERIODIC, None, stream)
                try:
                    rk.rk4_chain_set_kernel(h, kern)
                    st = st0.clone()
                    cp = torch.zeros_like(st) if prec == rk.RK4_FP32_KAHAN else None
                    wsb = rk.rk4_chain_workspace_bytes(h)
                    if kern == rk.RK4_KERNEL_AUTO:
                        rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_STAGED)
                        wsb = max(wsb, rk.rk4_chain_workspace_bytes(h))
                        rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_AUTO)
                    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
                    tiling = None
                    if kern == rk.RK4_KERNEL_AUTO:
                        tiling = rk.rk4_chain_autotune(h, st.clone(), cp.clone() if cp is not None else None, ws, 32)
                        tiling["kernel"] = {rk.RK4_KERNEL_STAGED: "standard", rk.RK4_KERNEL_BLOCKED: "blocked",
                                            rk.RK4_KERNEL_PERSISTENT: "persistent"}[rk.rk4_chain_get_kernel(h)]
                    elif kern != rk.RK4_KERNEL_STAGED:
                        if p <= 22 or (pname, sname) not in tuned:
                            tiling = rk.rk4_chain_autotune(h, st.clone(), cp.clone() if cp is not None else None,
                                                           ws, 32)
                            tuned[(pname, sname)] = tiling
                        else:
                            tiling = tuned[(pname, sname)]
                            rk.rk4_chain_set_tiling(h, tiling["block"], tiling["v"], tiling["k"])
                    # about 2^31 site-steps per measurement (at least 32 steps)
                    nsteps = max(32, min(4096, (1 << 31) // n))
                    if kern == rk.RK4_KERNEL_STAGED:
                        nsteps = max(8, nsteps // 4)
                    rk.rk4_chain_integrate(h, st, cp, ws, nsteps)  # warm-up, graph capture
                    el = min(time_integrate(rk, h, st, cp, ws, nsteps, 1, torch) for _ in range(3))
                    print(json.dumps({"N": n, "precision": pname, "scheme": sname, "site_steps_per_s": n * nsteps / el,
                                      "steps": nsteps, "tiling": tiling,
                                      "state_MB": n * D * (8 if prec == rk.RK4_FP64 else 4) / 1e6}), flush=True)
                    del st, cp, ws
                finally:
                    rk.rk4_chain_destroy(h)
            del st0
    return 0


def tiling_sweep(args):
    """The cluster-size study (Sec. 3.2.1, the paper's granularity dependence) on the N = 2^24
    periodic Roessler chain: for tile widths W = block x v from 256 to 8192 sites and k = 1, 2,
    4, 8 steps per launch (G = W - 8k interior sites), the fastest (block, v) realising W, FP64
    and FP32-Kahan.  Cells no block shape can realise (registers or shared memory per block)
    are printed with "infeasible" and the reason.  One JSON object per cell."""
    import torch
    import paper_1412_0544_gb300 as rk
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = N_SITES
    for prec, pname in ((rk.RK4_FP64, "fp64"), (rk.RK4_FP32_KAHAN, "fp32_kahan")):
        dtype = torch.float64 if prec == rk.RK4_FP64 else torch.float32
        h = rk.rk4_chain_create(rk.RK4_ROESSLER, prec, n, DT, rk.RK4_PERIODIC, None, stream)
        try:
            rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_BLOCKED)
            st = torch.empty((n, D), dtype=dtype, device="cuda")
            rk.rk4_fill_uniform(st, n * D, SEED, 0, prec, stream)
            cp = torch.zeros_like(st) if prec == rk.RK4_FP32_KAHAN else None
            ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
            for W in (256, 512, 1024, 2048, 4096, 8192):
                for k in (1, 2, 4, 8):
                    best, tried, reasons = None, [], []
                    for v in (1, 2, 4, 8):
                        block = W // v
                        if block < 64 or block > 1024 or block % 32:
                            reasons.append(f"v={v}: block {block} outside 64..1024")
                            continue
                        try:
                            rk.rk4_chain_set_tiling(h, block, v, k)
                        except rk.RK4Error:
                            reasons.append(f"v={v}: block {block} exceeds the kernel's limit (registers or shared memory)")
                            continue
                        nsteps = 16 * k if prec == rk.RK4_FP32_KAHAN else 8 * k
                        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)  # warm-up, graph capture
                        el = min(time_integrate(rk, h, st, cp, ws, nsteps, 1, torch) for _ in range(2))
                        sps = n * nsteps / el
                        tried.append({"block": block, "v": v, "site_steps_per_s": sps})
                        if best is None or sps > best["site_steps_per_s"]:
                            best = tried[-1]
                    line = {"precision": pname, "N": n, "W": W, "k": k, "G": W - 8 * k}
                    if best is None:
                        line.update({"infeasible": True, "reason": "; ".join(reasons)})
                    else:
                        line.update({"best": best, "tried": tried})
                    print(json.dumps(line), flush=True)
        finally:
            rk.rk4_chain_destroy(h)
    return 0


# Dormand and Prince (1980) RK5(4)7M, fifth-order weights, used with a fixed step
DOPRI5_A = np.array([
    [0, 0, 0, 0, 0, 0, 0],
    [1 / 5, 0, 0, 0, 0, 0, 0],
    [3 / 40, 9 / 40, 0, 0, 0, 0, 0],
    [44 / 45, -56 / 15, 32 / 9, 0, 0, 0, 0],
    [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729, 0, 0, 0],
    [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656, 0, 0],
    [35 / 384, 0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0]])
DOPRI5_B = np.array([35 / 384, 0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0])


def generic_fp_ops(A, b, D, slope_ops, kahan):
    """Algorithmic floating-point instructions per site-step of the generic scheme: the slopes
    and stage states of the stages the result needs (a stage is needed when its weight b_m is
    nonzero or a needed later stage uses it; Dormand-Prince 5's seventh stage, with b_7 = 0,
    is not), the weighted sum and the update (FP32-Kahan: 4 per component instead of 1)."""
    s = len(b)
    A = np.tril(np.asarray(A, dtype=float), -1)
    needed = {m for m in range(s) if b[m] != 0}
    for j in range(s - 1, -1, -1):
        if j in needed:
            needed |= {m for m in range(j) if A[j][m] != 0}
    return (sum(int(np.count_nonzero(A[j])) for j in needed) * D + len(needed) * slope_ops
            + int(np.count_nonzero(b)) * D + (4 if kahan else 1) * D)


def variant_extra(rk, torch, stream, precision, *, generic=False, het=False, n=N_SITES, nsteps=200):
    """The widened scheme on the same N = 2^24 periodic Roessler chain: Dormand-Prince 5 with
    second-neighbour coupling (generic kernel, halo 12 sites per side per step: six needed
    stages x range 2), or a heterogeneous chain with per-site parameters (Eq. (1))."""
    import chain_inputs as ci
    fp32 = precision == rk.RK4_FP32_KAHAN
    dtype = torch.float32 if fp32 else torch.float64
    h = rk.rk4_chain_create(rk.RK4_ROESSLER, precision, n, DT, rk.RK4_PERIODIC, None, stream)
    try:
        sp = None
        if generic:
            rk.rk4_chain_set_tableau(h, DOPRI5_A, DOPRI5_B)
            rk.rk4_chain_set_coupling2(h, 0.5)
            ops = generic_fp_ops(DOPRI5_A, DOPRI5_B, D, 10, fp32)
        if het:
            u = ci.uniform01(SEED, 9, 0, 4 * n).reshape(n, 4)
            sp = torch.from_numpy(np.stack([0.15 + 0.1 * u[:, 0], 0.8 + 0.4 * u[:, 1], 8.0 + 2.0 * u[:, 2],
                                            0.5 + 1.5 * u[:, 3]], axis=1)).to(dtype).cuda()
            rk.rk4_chain_set_site_params(h, sp)
            ops = FP32K_INST_PER_SITE_STEP if fp32 else FP64_INST_PER_SITE_STEP
        st = torch.empty((n, D), dtype=dtype, device="cuda")
        rk.rk4_fill_uniform(st, n * D, SEED, 0, precision, stream)
        cp = torch.zeros_like(st) if fp32 else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        best = rk.rk4_chain_autotune(h, st.clone(), cp.clone() if cp is not None else None, ws, 16)
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)  # warm-up with the timed step count (graph cached)
        el = time_integrate(rk, h, st, cp, ws, nsteps, 1, torch)
        sps = n * nsteps / el
        peak = FP32_INST_PEAK if fp32 else FP64_INST_PEAK
        return {"value": sps, "unit": "site-steps/s", "N": n, "steps": nsteps, "tiling": best,
                "fp_inst_per_site_step": ops, "pipe_frac_of_measured": sps * ops / peak,
                "kernel_hash": kernel_hash(files=GENERIC_SOURCES if generic else BLOCKED_SOURCES),
                "scheme": ("Dormand-Prince 5 (7 stages) + second-neighbour coupling" if generic
                           else "heterogeneous chain, per-site a, b, c, kappa")}
    finally:
        rk.rk4_chain_destroy(h)


def domain_extra(rk, torch, stream, precision, nparts=4, ghost=32, n=N_SITES, nsteps=200):
    """The N = 2^24 periodic Roessler chain split into `nparts` sub-domains with `ghost` sites of
    ghost zone per side (classical RK4 reaches 4 sites per step: ghost / 4 steps between
    device-to-device ghost exchanges), against the undivided chain at the same tiling."""
    fp32 = precision == rk.RK4_FP32_KAHAN
    dtype = torch.float32 if fp32 else torch.float64
    d = rk.rk4_domain_create(rk.RK4_ROESSLER, precision, n, DT, rk.RK4_PERIODIC, nparts, ghost, None, None, stream)
    h = rk.rk4_chain_create(rk.RK4_ROESSLER, precision, n, DT, rk.RK4_PERIODIC, None, stream)
    try:
        tiling = rk.rk4_chain_get_tiling(rk.rk4_domain_chain(d))
        # the undivided chain with the same launch shape (k steps per launch)
        rk.rk4_chain_set_tiling(h, tiling["block"], tiling["v"], tiling["k"])
        cst = torch.empty((n, D), dtype=dtype, device="cuda")
        rk.rk4_fill_uniform(cst, n * D, SEED, 0, precision, stream)
        ccp = torch.zeros_like(cst) if fp32 else None
        rows, _ = rk.rk4_domain_shape(d)
        st = torch.empty((rows, D), dtype=dtype, device="cuda")
        cp = torch.zeros_like(st) if fp32 else None
        ws = torch.empty(rk.rk4_domain_workspace_bytes(d), dtype=torch.uint8, device="cuda")
        rk.rk4_domain_scatter(d, cst, ccp, st, cp)
        rk.rk4_domain_integrate(d, st, cp, ws, nsteps)  # warm-up with the timed step count (graphs)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        rk.rk4_domain_integrate(d, st, cp, ws, nsteps)
        e1.record(s)
        e1.synchronize()
        el = e0.elapsed_time(e1) / 1e3
        wsw = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_integrate(h, cst, ccp, wsw, nsteps)  # warm-up with the timed step count (graph cached)
        el_whole = time_integrate(rk, h, cst, ccp, wsw, nsteps, 1, torch)
        return {"value": n * nsteps / el, "unit": "site-steps/s", "N": n, "steps": nsteps, "parts": nparts,
                "ghost": ghost, "steps_per_exchange": ghost // 4, "tiling": tiling,
                "undivided_same_tiling": n * nsteps / el_whole, "ratio_to_undivided": el_whole / el}
    finally:
        rk.rk4_chain_destroy(h)
        rk.rk4_domain_destroy(d)


PAPER_N, PAPER_STEPS, PAPER_TRIALS = 1 << 20, 50, 10


def paper_workload_extra(rk, torch, stream, precision):
    """The paper's own benchmark (Sec. 3.2): a periodic Roessler chain of N = 2^20 from random
    initial conditions, T = 50 RK4 steps of dt = 0.01, performance = T / t_wall in RK4 steps/s,
    the best of 10 trials.  The 25 MB FP64 state fits in the 129 MB L2, so this measures the
    L2-resident regime.  The paper's CPU figures (one Xeon core) are context only."""
    fp32 = precision == rk.RK4_FP32_KAHAN
    dtype = torch.float32 if fp32 else torch.float64
    n = PAPER_N
    h = rk.rk4_chain_create(rk.RK4_ROESSLER, precision, n, DT, rk.RK4_PERIODIC, None, stream)
    try:
        st = torch.empty((n, D), dtype=dtype, device="cuda")
        rk.rk4_fill_uniform(st, n * D, SEED, 0, precision, stream)
        cp = torch.zeros_like(st) if fp32 else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        best = rk.rk4_chain_autotune(h, st.clone(), cp.clone() if cp is not None else None, ws, 16)
        for _ in range(3):
            rk.rk4_chain_integrate(h, st, cp, ws, PAPER_STEPS)
        trials = [time_integrate(rk, h, st, cp, ws, PAPER_STEPS, 1, torch) for _ in range(PAPER_TRIALS)]
        t = min(trials)
        return {"value": PAPER_STEPS / t, "unit": "RK4 steps/s", "site_steps_per_s": n * PAPER_STEPS / t,
                "N": n, "steps": PAPER_STEPS, "trials": PAPER_TRIALS, "median_steps_per_s": PAPER_STEPS /
                sorted(trials)[len(trials) // 2], "tiling": best, "l2": "state fits in L2",
                "paper_context": "one Xeon E5 core (Sec. 3.2.1): standard < 30 steps/s, cache-optimised + SIMD "
                                 "about 3x that"}
    finally:
        rk.rk4_chain_destroy(h)


def paper_workload_oracle(trials: int = 5) -> dict:
    """The serial C oracle on one host core under the same protocol (best of `trials`)."""
    import chain_inputs as ci
    import oracle
    y0 = ci.uniform_state(PAPER_N, D, seed=SEED)
    oracle.load()
    ts = []
    for _ in range(trials):
        t0 = time.perf_counter()
        oracle.rk4_integrate(y0, oracle.ROESSLER, oracle.PERIODIC, DT, PAPER_STEPS)
        ts.append(time.perf_counter() - t0)
    return {"value": PAPER_STEPS / min(ts), "unit": "RK4 steps/s", "cores": 1, "kind": "oracle",
            "trials": trials}


def harmonic_energy_extra(rk, torch, stream, n=N_SITES, nsteps=NSTEPS, kappa=1.0, omega0=1.0):
    """Energy behaviour where the chain is Hamiltonian: the periodic harmonic chain (D = 2),
    N = 2^24, 1000 steps, FP64 and FP32-Kahan; the measured relative drift of the FP64
    energy reduction next to RK4's exact per-mode energy factor rho(h)^n summed over the
    Fourier modes of the initial state."""
    out = {}
    y0 = None
    for precision, name in ((rk.RK4_FP64, "fp64"), (rk.RK4_FP32_KAHAN, "fp32_kahan")):
        fp32 = precision == rk.RK4_FP32_KAHAN
        h = rk.rk4_chain_create(rk.RK4_HARMONIC, precision, n, DT, rk.RK4_PERIODIC,
                                dict(kappa=kappa, omega0=omega0), stream)
        try:
            st = torch.empty((n, 2), dtype=torch.float32 if fp32 else torch.float64, device="cuda")
            rk.rk4_fill_uniform(st, n * 2, SEED, 0, precision, stream)
            if y0 is None:
                y0 = st.double().cpu().numpy()
            cp = torch.zeros_like(st) if fp32 else None
            ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
            rk.rk4_chain_integrate(h, st, cp, ws, nsteps)  # warm-up with the timed step count (graph cached)
            rk.rk4_fill_uniform(st, n * 2, SEED, 0, precision, stream)
            if cp is not None:
                cp.zero_()
            e0 = rk.rk4_chain_energy(h, st, cp, ws)[0]
            el = time_integrate(rk, h, st, cp, ws, nsteps, 1, torch)
            e1 = rk.rk4_chain_energy(h, st, cp, ws)[0]
            out[name] = {"site_steps_per_s": n * nsteps / el, "E0": e0, "E_final": e1,
                         "rel_drift": (e1 - e0) / e0}
        finally:
            rk.rk4_chain_destroy(h)
    # RK4 multiplies each mode's energy by rho(h) = 1 - h^6/72 + h^8/576 per step (h = omega_m dt)
    m = np.arange(n)
    w = np.sqrt(omega0 ** 2 + 4.0 * kappa * np.sin(np.pi * m / n) ** 2)
    qh, ph = np.fft.fft(y0[:, 0]), np.fft.fft(y0[:, 1])
    em = 0.5 * (np.abs(ph) ** 2 + w ** 2 * np.abs(qh) ** 2) / n
    hm = w * DT
    rho = 1.0 - hm ** 6 / 72.0 + hm ** 8 / 576.0
    out["predicted_rel_drift"] = float(np.sum(em * rho ** nsteps) / np.sum(em) - 1.0)
    out["N"], out["steps"] = n, nsteps
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP32 and batch side measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-probe", action="store_true",
                    help="quote ALU rooflines against the stored peaks instead of running pipe_probe first")
    ap.add_argument("--tiling", default=None, help="block,v,k of the FP64 kernel instead of the autotuner's pick")
    ap.add_argument("--sweep", action="store_true", help="site-steps/s against chain length instead of the bench line")
    ap.add_argument("--sweep-min", type=int, default=10, help="log2 of the smallest N of --sweep")
    ap.add_argument("--sweep-max", type=int, default=27, help="log2 of the largest N of --sweep")
    ap.add_argument("--tiling-sweep", action="store_true",
                    help="site-steps/s against tile width and steps per launch instead of the bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return size_sweep(args)
    if args.tiling_sweep:
        return tiling_sweep(args)

    import torch

    from paper_1412_0544_gb300 import dist
    import paper_1412_0544_gb300 as rk

    rank, world, local = dist.env_rank()
    torch.cuda.set_device(local)  # before the process group, so NCCL binds this rank's GPU
    rank, world, local = dist.init("nccl")
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_GBS_FALLBACK))
    probe = probe_peaks() if rank == 0 and not args.no_probe else None

    # --- the workload: one chain per rank (independent replicas, weak scaling) -------
    n, nsteps = N_HEAD, NSTEPS_HEAD
    h = rk.rk4_chain_create(rk.RK4_ROESSLER, rk.RK4_FP64, n, DT, rk.RK4_FIXED, None, stream)
    st = torch.empty((n, D), dtype=torch.float64, device="cuda")
    rk.rk4_fill_uniform(st, n * D, SEED, 0, rk.RK4_FP64, stream)
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    if args.tiling:
        rk.rk4_chain_set_tiling(h, *[int(x) for x in args.tiling.split(",")])
        tiling = rk.rk4_chain_get_tiling(h)
    else:
        tiling = rk.rk4_chain_autotune(h, st.clone(), None, ws, 16)
    plan_launches = -(-nsteps // tiling["k"])
    plan_launches += plan_launches % 2  # the plan keeps an even launch count when it can

    def one_step():
        rk.rk4_chain_integrate(h, st, None, ws, nsteps)
        return rk.rk4_chain_energy(h, st, None, ws)[0]  # synchronises; checks for NaN/inf

    for _ in range(args.warmup):
        one_step()
    dist.barrier()
    torch.cuda.synchronize()
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0, e1 = marks[0], marks[-1]
    with ClockSampler(local) as clocks:
        e0.record(stream)
        for i in range(args.steps):
            norm = one_step()
            marks[i + 1].record(stream)
        e1.synchronize()
    step_ms = sorted(marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps))
    torch.cuda.synchronize()
    dist.barrier()
    el = dist.max_over_ranks(e0.elapsed_time(e1) / 1e3)
    site_steps = float(n) * nsteps * args.steps * world
    value = site_steps / el

    # kernel-only timing of the blocked kernel for the roofline (same stream, events)
    reps = 2
    el_k = time_integrate(rk, h, st, None, ws, nsteps, reps, torch)
    launch_s = el_k / (reps * plan_launches)
    sps_k = n * nsteps * reps / el_k
    achieved_inst = sps_k * FP64_INST_PER_SITE_STEP / 1e9  # G FP64 instructions/s
    khash = kernel_hash()
    traffic = traffic_per_launch(khash, tiling, n)
    roofline = {"bound": "alu", "achieved": achieved_inst, "peak": FP64_INST_PEAK / 1e9,
                "unit": "G FP64 inst/s", "frac": achieved_inst * 1e9 / FP64_INST_PEAK,
                "traffic": traffic, "kernel": "k_blocked<double, Roessler>",
                "per_unit": "49 FP64 instructions per interior site-step",
                "launch_ms": launch_s * 1e3,
                "peak_source": PEAK_SOURCE + " (DFMA issue rate; all 49 operations of the step can issue "
                                             "as DFMA)",
                "hbm_frac_effective_state": sps_k * 2 * D * 8 / 1e9 / hbm_peak,
                # DRAM bandwidth the kernel draws: ncu's bytes per launch over this run's launch time
                "dram_GBs": traffic / launch_s / 1e9 if traffic else None}
    if probe and "rk4_fp64_regs_inst_per_s" in probe:
        # the same RK4 instruction stream on register-resident sites (no loads, exchange or
        # barriers): the most this instruction mix reaches on the FP64 pipe
        arith_rate = float(probe["rk4_fp64_regs_inst_per_s"])
        roofline["arithmetic_only_rate"] = arith_rate / 1e9
        roofline["frac_of_arithmetic_only"] = achieved_inst * 1e9 / arith_rate
    if probe and "rk4_fp64_regs_smem_roundtrip_inst_per_s" in probe:
        # the same stream with a tile kernel's per-stage shared-memory exchange and barrier
        xrate = float(probe["rk4_fp64_regs_smem_roundtrip_inst_per_s"])
        roofline["arithmetic_with_exchange_rate"] = xrate / 1e9
        roofline["frac_of_arithmetic_with_exchange"] = achieved_inst * 1e9 / xrate

    # --- end to end through the C ABI with host buffers ------------------------------
    host = torch.empty((n, D), dtype=torch.float64).pin_memory()
    host.copy_(st.cpu())
    dev2 = torch.empty_like(st)
    rk.rk4_chain_integrate_host(h, host, None, dev2, None, ws, nsteps)  # warm
    dist.barrier()
    e2e_steps = 2
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(local) as e2e_clocks:
        t0 = time.perf_counter()
        ev[0].record(stream)
        for _ in range(e2e_steps):
            rk.rk4_chain_integrate_host(h, host, None, dev2, None, ws, nsteps)
        ev[1].record(stream)
        ev[1].synchronize()
        el_e2e = dist.max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": float(n) * nsteps * e2e_steps * world / el_e2e, "unit": "site-steps/s",
           "h2d_bytes_per_step": n * D * 8, "d2h_bytes_per_step": n * D * 8,
           "api": "rk4_chain_integrate_host (pinned host state in, result out)",
           "device_s_per_step": ev[0].elapsed_time(ev[1]) / 1e3 / e2e_steps,
           "wall_s_per_step": el_e2e / e2e_steps, "clocks": e2e_clocks.summary()}
    del host, dev2

    extras = {}
    if world > 1:
        # per-GPU side measurements add nothing to a weak-scaling line and would hold every GPU
        extras["extras"] = "skipped for n_gpus > 1 (run with one GPU)"
    elif not args.no_extras:
        extras["periodic_fp64_2e24_1000steps"] = periodic_fp64_extra(rk, torch, stream)
        extras["fp32_kahan_2e27"] = fp32_kahan_extra(rk, torch, stream)
        extras["batch_fp64"] = batch_extra(rk, torch, stream, rk.RK4_FP64)
        extras["batch_fp32_kahan"] = batch_extra(rk, torch, stream, rk.RK4_FP32_KAHAN)
        extras["harmonic_energy"] = harmonic_energy_extra(rk, torch, stream)
        extras["generic_dopri5_nnn_fp64"] = variant_extra(rk, torch, stream, rk.RK4_FP64, generic=True)
        extras["generic_dopri5_nnn_fp32_kahan"] = variant_extra(rk, torch, stream, rk.RK4_FP32_KAHAN, generic=True,
                                                                nsteps=1000)
        extras["heterogeneous_fp64"] = variant_extra(rk, torch, stream, rk.RK4_FP64, het=True)
        extras["heterogeneous_fp32_kahan"] = variant_extra(rk, torch, stream, rk.RK4_FP32_KAHAN, het=True,
                                                           nsteps=1000)
        extras["paper_workload_2e20_fp64"] = paper_workload_extra(rk, torch, stream, rk.RK4_FP64)
        extras["paper_workload_2e20_fp32_kahan"] = paper_workload_extra(rk, torch, stream, rk.RK4_FP32_KAHAN)
        extras["domain_4parts_fp64"] = domain_extra(rk, torch, stream, rk.RK4_FP64)
        extras["domain_4parts_fp32_kahan"] = domain_extra(rk, torch, stream, rk.RK4_FP32_KAHAN, ghost=64, nsteps=1000)
    rk.rk4_chain_destroy(h)

    out = None
    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value, "unit": "site-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "step_ms": {"min": step_ms[0], "median": step_ms[len(step_ms) // 2], "max": step_ms[-1]},
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sites": n, "rk4_steps_per_step": nsteps,
                       "dt": DT, "boundary": BC_HEAD, "tiling": tiling, "l2": "inputs larger than L2 (3.2 GB state)",
                       "parallelism": f"replicas x{world}", "final_half_norm2": float(norm)},
            "roofline": roofline,
            "effective_state_GBs": value / world * 2 * D * 8 / 1e9,
            "pct_hbm_roofline_effective": 100.0 * value / world * 2 * D * 8 / 1e9 / hbm_peak,
            "clocks": clocks.summary(),
            "e2e": e2e,
            "gpu_launches": args.steps * (plan_launches + 2),
            "kernel_hash": khash,
            "alu_peaks": {"fp64_dfma_per_s": FP64_INST_PEAK, "fp32_fma_lanes_per_s": FP32_INST_PEAK,
                          "source": PEAK_SOURCE, "probe": probe},
        }
        out.update(extras)
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline()
            out["cpu_baseline"]["host"] = host_info()
            if "paper_workload_2e20_fp64" in out:
                out["paper_workload_2e20_fp64"]["oracle_1core"] = paper_workload_oracle()
        print(json.dumps(out))
    dist.barrier()
    return 0


if __name__ == "__main__":
    sys.exit(main())
