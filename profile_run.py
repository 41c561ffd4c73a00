"""A short, fixed workload for profiler captures (ncu): fills a chain (or a batch) and advances
it a given number of RK4 steps with a fixed tiling, then exits.  Nothing is timed here.

    python profile_run.py --precision fp64 --n 16777216 --steps 4 --tiling 256,4,2
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--model", choices=["roessler", "harmonic"], default="roessler")
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--bc", choices=["periodic", "fixed"], default="periodic")
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--tiling", default="256,4,1")
    ap.add_argument("--kernel", choices=["blocked", "staged", "persistent"], default="blocked")
    ap.add_argument("--batch", type=int, default=0, help="integrate this many uneven chains instead of one")
    ap.add_argument("--parts", type=int, default=0, help="integrate this many equal periodic chains of n / parts")
    ap.add_argument("--tableau", choices=["rk4", "dopri5"], default="rk4",
                    help="dopri5: the generic kernels with Dormand and Prince's 7-stage tableau")
    ap.add_argument("--kappa2", type=float, default=0.0, help="second-neighbour coupling (generic kernels)")
    ap.add_argument("--het", action="store_true",
                    help="heterogeneous chain: per-site a, b, c, kappa drawn as in bench.py (Eq. (1))")
    args = ap.parse_args()

    import torch

    import chain_inputs as ci
    import paper_1412_0544_gb300 as rk

    prec = rk.RK4_FP64 if args.precision == "fp64" else rk.RK4_FP32_KAHAN
    model = rk.RK4_ROESSLER if args.model == "roessler" else rk.RK4_HARMONIC
    D = 3 if model == rk.RK4_ROESSLER else 2
    if args.batch:
        lengths, kappa, bcs = ci.batch_spec(args.batch)
        h = rk.rk4_batch_create(model, prec, lengths, kappa, bcs, 0.01)
        total = int(lengths.sum())
    elif args.parts:
        import numpy as np
        lengths = np.full(args.parts, args.n // args.parts, dtype=np.int64)
        h = rk.rk4_batch_create(model, prec, lengths, np.ones(args.parts), np.zeros(args.parts, dtype=np.int8), 0.01)
        total = int(lengths.sum())
    else:
        h = rk.rk4_chain_create(model, prec, args.n, 0.01, rk.RK4_PERIODIC if args.bc == "periodic" else rk.RK4_FIXED)
        total = args.n
    kern = {"blocked": rk.RK4_KERNEL_BLOCKED, "staged": rk.RK4_KERNEL_STAGED,
            "persistent": rk.RK4_KERNEL_PERSISTENT}[args.kernel]
    rk.rk4_chain_set_kernel(h, kern)
    if args.tableau == "dopri5":
        import bench
        rk.rk4_chain_set_tableau(h, bench.DOPRI5_A, bench.DOPRI5_B)
    if args.kappa2:
        rk.rk4_chain_set_coupling2(h, args.kappa2)
    if args.het:
        import numpy as np
        import bench
        u = ci.uniform01(bench.SEED, 9, 0, 4 * total).reshape(total, 4)
        sp = torch.from_numpy(np.stack([0.15 + 0.1 * u[:, 0], 0.8 + 0.4 * u[:, 1], 8.0 + 2.0 * u[:, 2],
                                        0.5 + 1.5 * u[:, 3]], axis=1))
        sp = sp.to(torch.float64 if prec == rk.RK4_FP64 else torch.float32).cuda()
        rk.rk4_chain_set_site_params(h, sp)
    rk.rk4_chain_set_tiling(h, *[int(x) for x in args.tiling.split(",")])
    rk.rk4_chain_set_option(h, rk.RK4_OPT_GRAPHS, 0)
    dtype = torch.float64 if prec == rk.RK4_FP64 else torch.float32
    st = torch.empty((total, D), dtype=dtype, device="cuda")
    rk.rk4_fill_uniform(st, total * D, ci.DEFAULT_SEED, 0, prec)
    cp = torch.zeros_like(st) if prec == rk.RK4_FP32_KAHAN else None
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    rk.rk4_chain_integrate(h, st, cp, ws, args.steps)
    torch.cuda.synchronize()
    print("tiling", rk.rk4_chain_get_tiling(h), "sites", total)
    rk.rk4_chain_destroy(h)


if __name__ == "__main__":
    main()
