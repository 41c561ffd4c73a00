"""Helpers shared by the GPU tests: run the CUDA library through the C ABI on numpy inputs."""
from __future__ import annotations

import numpy as np
import torch

import paper_1412_0544_gb300 as rk


def to_dev(a: np.ndarray, dtype) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def gpu_run(y0, *, model=rk.RK4_ROESSLER, precision=rk.RK4_FP64, bc=rk.RK4_PERIODIC, nsteps=1, dt=0.01,
            params=None, kernel=rk.RK4_KERNEL_AUTO, tiling=None, lengths=None, kappas=None, bcs=None,
            graphs=True, comp0=None, return_comp=False, chunks=None):
    """Integrate y0 ([N, D] numpy) on the GPU; returns the result as float64 numpy (and the
    Kahan compensation when asked).  ``chunks`` splits nsteps into several calls."""
    fp32 = precision == rk.RK4_FP32_KAHAN
    dtype = torch.float32 if fp32 else torch.float64
    if lengths is not None:
        h = rk.rk4_batch_create(model, precision, lengths, kappas, bcs, dt, params)
    else:
        h = rk.rk4_chain_create(model, precision, y0.shape[0], dt, bc, params)
    try:
        if kernel != rk.RK4_KERNEL_AUTO:
            rk.rk4_chain_set_kernel(h, kernel)
        if tiling is not None:
            rk.rk4_chain_set_tiling(h, *tiling)
        if not graphs:
            rk.rk4_chain_set_option(h, rk.RK4_OPT_GRAPHS, 0)
        st = to_dev(y0, dtype)
        cp = None
        if fp32:
            cp = torch.zeros_like(st) if comp0 is None else to_dev(comp0, dtype)
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        for n in (chunks or [nsteps]):
            rk.rk4_chain_integrate(h, st, cp, ws, n)
        torch.cuda.synchronize()
        assert rk.rk4_chain_status(h, ws) == rk.RK4_OK
        out = st.double().cpu().numpy()
        if return_comp:
            return out, (cp.double().cpu().numpy() if cp is not None else None)
        return out
    finally:
        rk.rk4_chain_destroy(h)
