"""A thin convenience wrapper: one handle plus a torch-owned workspace.

It only allocates device memory through torch and forwards to the C ABI; the integration
itself runs in librk4chain.so.
"""
from __future__ import annotations

import numpy as np

from . import (RK4_FP32_KAHAN, RK4_FP64, RK4_KERNEL_AUTO, RK4_PERIODIC, RK4_ROESSLER, rk4_batch_create,
               rk4_chain_create, rk4_chain_destroy, rk4_chain_energy, rk4_chain_get_tiling,
               rk4_chain_integrate, rk4_chain_set_kernel, rk4_chain_set_tiling, rk4_chain_shape,
               rk4_chain_status, rk4_chain_workspace_bytes)


class Chain:
    """One chain (``n``) or a batch (``lengths``, ``kappas``, ``bcs``) on the current CUDA device.

    ``state`` tensors are [total_sites, D] contiguous float64 (FP64) or float32 (FP32-Kahan);
    ``comp`` is the matching Kahan compensation (FP32 only).
    """

    def __init__(self, n=None, *, lengths=None, kappas=None, bcs=None, model=RK4_ROESSLER, precision=RK4_FP64,
                 bc=RK4_PERIODIC, dt=0.01, params=None, kernel=RK4_KERNEL_AUTO, tiling=None, stream=None):
        import torch
        self._torch = torch
        self.stream = stream
        if lengths is not None:
            self.h = rk4_batch_create(model, precision, lengths, kappas, bcs, dt, params, stream)
            self.nchains = len(lengths)
        else:
            self.h = rk4_chain_create(model, precision, n, dt, bc, params, stream)
            self.nchains = 1
        self.model, self.precision = model, precision
        self.total, self.D = rk4_chain_shape(self.h)
        self.dtype = torch.float32 if precision == RK4_FP32_KAHAN else torch.float64
        self._ws = None
        if kernel != RK4_KERNEL_AUTO:
            rk4_chain_set_kernel(self.h, kernel)
        if tiling is not None:
            rk4_chain_set_tiling(self.h, *tiling)

    # -- workspace -----------------------------------------------------------------------
    def workspace(self):
        need = rk4_chain_workspace_bytes(self.h)
        if self._ws is None or self._ws.numel() < need:
            self._ws = self._torch.empty(need, dtype=self._torch.uint8, device="cuda")
        return self._ws

    def set_kernel(self, kernel: int):
        rk4_chain_set_kernel(self.h, kernel)

    def set_tiling(self, block: int, v: int = 0, k: int = 0):
        rk4_chain_set_tiling(self.h, block, v, k)

    @property
    def tiling(self) -> dict:
        return rk4_chain_get_tiling(self.h)

    # -- buffers -------------------------------------------------------------------------
    def new_state(self, values=None):
        torch = self._torch
        if values is None:
            return torch.zeros((self.total, self.D), dtype=self.dtype, device="cuda")
        t = torch.as_tensor(np.ascontiguousarray(values)).to(self.dtype)
        return t.reshape(self.total, self.D).contiguous().cuda()

    def new_comp(self):
        if self.precision != RK4_FP32_KAHAN:
            return None
        return self._torch.zeros((self.total, self.D), dtype=self.dtype, device="cuda")

    # -- operations ----------------------------------------------------------------------
    def integrate(self, state, comp, nsteps: int) -> float:
        return rk4_chain_integrate(self.h, state, comp, self.workspace(), nsteps)

    def energy(self, state, comp=None) -> np.ndarray:
        return rk4_chain_energy(self.h, state, comp, self.workspace())

    def status(self) -> int:
        return rk4_chain_status(self.h, self.workspace())

    def autotune(self, state, comp, probe_steps: int = 16, *, cache: str | None = None, scheme: str = "rk4") -> dict:
        """Tunes on copies of state/comp (the tuner advances the buffers it is given).  With a
        cache file (``cache`` or RK4CHAIN_TUNE_CACHE) a stored choice for the same GPU and
        workload is applied instead of tuning (tune_cache); ``scheme`` tags the workload when a
        tableau, second-neighbour coupling or site parameters were set on the handle."""
        from . import tune_cache
        s = state.clone()
        c = comp.clone() if comp is not None else None
        key = tune_cache.make_key(self._torch.cuda.get_device_name(), self.model, self.precision, self.nchains,
                                  self.total, scheme)
        return tune_cache.autotune(self.h, s, c, self.workspace(), key, probe_steps=probe_steps, path=cache)

    def close(self):
        if self.h is not None:
            rk4_chain_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
