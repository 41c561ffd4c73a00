"""Checkpoint and resume of an integration: the state (and, for FP32-Kahan, the compensation,
which is part of the integrator's state), the handle's clock (t0 and steps taken) and a JSON
header describing the chain, in one ``.npz`` file.

Because every scheme performs the same per-site operations, integrating a steps, saving,
loading into a fresh handle and integrating b more steps is bit-identical to integrating a + b
steps in one go.
"""
from __future__ import annotations

import json

import numpy as np

FORMAT = "rk4chain-checkpoint-1"


def save(path: str, state, comp=None, *, t0: float = 0.0, nstep: int = 0, **header) -> None:
    """Write state / comp (torch tensors or numpy arrays) and the clock to ``path``."""
    st = _to_numpy(state)
    arrays = {"state": st}
    if comp is not None:
        arrays["comp"] = _to_numpy(comp)
    meta = dict(header)
    meta.update({"format": FORMAT, "t0": float(t0), "nstep": int(nstep), "dtype": str(st.dtype),
                 "shape": list(st.shape)})
    arrays["header"] = np.frombuffer(json.dumps(meta, sort_keys=True).encode(), dtype=np.uint8)
    with open(path, "wb") as f:
        np.savez(f, **arrays)


def load(path: str):
    """Returns (state, comp or None, header dict) as numpy arrays."""
    with np.load(path) as z:
        meta = json.loads(bytes(z["header"]).decode())
        if meta.get("format") != FORMAT:
            raise ValueError(f"{path}: not a {FORMAT} file")
        state = z["state"].copy()
        comp = z["comp"].copy() if "comp" in z.files else None
    if list(state.shape) != meta["shape"] or str(state.dtype) != meta["dtype"]:
        raise ValueError(f"{path}: header does not match the stored state")
    return state, comp, meta


def save_handle(path: str, rk, h, state, comp=None, **header) -> None:
    """Checkpoint a handle's state and clock (rk: the binding module)."""
    t0, n = rk.rk4_chain_get_clock(h)
    save(path, state, comp, t0=t0, nstep=n, **header)


def restore_handle(path: str, rk, h, device="cuda"):
    """Load a checkpoint into device tensors for handle h and restore its clock; returns
    (state, comp or None, header)."""
    import torch
    state, comp, meta = load(path)
    rk.rk4_chain_set_clock(h, meta["t0"], meta["nstep"])
    st = torch.from_numpy(state).to(device)
    cp = torch.from_numpy(comp).to(device) if comp is not None else None
    return st, cp, meta


def _to_numpy(x) -> np.ndarray:
    if hasattr(x, "detach"):
        return x.detach().cpu().numpy()
    return np.ascontiguousarray(x)
