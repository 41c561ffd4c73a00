"""Python binding of librk4chain.so (include/rk4chain.h): classical RK4 on long
nearest-neighbour chains (Mulansky, arXiv:1412.0544) as hand-written CUDA for GB300.

This module only marshals arguments: every step of the integration runs in the CUDA library.
Functions keep the C names and return values instead of out-parameters; a nonzero return code
raises :class:`RK4Error`.  Buffers may be torch tensors (their data pointer and size are
passed) or plain integer device/host addresses.  There is no CPU fallback: if the library is
not built, importing this package raises ``ImportError``.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RK4CHAIN_LIBRARY selects another build of the same ABI (for example librk4chain_debug.so,
# whose kernels check every memory range they touch).
LIB_PATH = os.environ.get("RK4CHAIN_LIBRARY") or os.path.join(_HERE, "librk4chain.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "rk4chain.h")

RK4_OK, RK4_EINVAL, RK4_ENOMEM_WS, RK4_ECUDA, RK4_ENONFINITE, RK4_ETIMEOUT, RK4_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
RK4_EBOUNDS = -7
RK4_ROESSLER, RK4_HARMONIC = 0, 1
RK4_FP64, RK4_FP32_KAHAN = 0, 1
RK4_PERIODIC, RK4_FIXED = 0, 1
RK4_KERNEL_AUTO, RK4_KERNEL_STAGED, RK4_KERNEL_BLOCKED, RK4_KERNEL_PERSISTENT = 0, 1, 2, 3
RK4_OPT_GRAPHS, RK4_OPT_TIMEOUT_NS = 0, 1


class RK4Error(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {rk4_strerror(code)} ({code})")
        self.code = code


class rk4_params(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
                ("kappa", ctypes.c_double), ("omega0", ctypes.c_double)]


class rk4_tiling(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("v", ctypes.c_int), ("k", ctypes.c_int), ("G", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built: run `python paper_1412_0544_gb300/build.py` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, c_int, sz, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)
    H = ctypes.c_void_p
    sig = {
        "rk4_params_default": (None, [ctypes.POINTER(rk4_params)]),
        "rk4_chain_create": (c_int, [ctypes.POINTER(H), c_int, c_int, i64, ctypes.c_double, c_int,
                                     ctypes.POINTER(rk4_params), vp]),
        "rk4_batch_create": (c_int, [ctypes.POINTER(H), c_int, c_int, c_int, ctypes.POINTER(i64), dp,
                                     ctypes.POINTER(ctypes.c_int8), ctypes.c_double, ctypes.POINTER(rk4_params), vp]),
        "rk4_chain_workspace_bytes": (c_int, [H, ctypes.POINTER(sz)]),
        "rk4_chain_shape": (c_int, [H, ctypes.POINTER(i64), ctypes.POINTER(c_int)]),
        "rk4_chain_set_kernel": (c_int, [H, c_int]),
        "rk4_chain_set_tiling": (c_int, [H, c_int, c_int, c_int]),
        "rk4_chain_get_tiling": (c_int, [H, ctypes.POINTER(rk4_tiling)]),
        "rk4_chain_get_kernel": (c_int, [H, ctypes.POINTER(c_int)]),
        "rk4_chain_autotune": (c_int, [H, vp, vp, vp, sz, c_int, ctypes.POINTER(rk4_tiling)]),
        "rk4_chain_step": (c_int, [H, vp, vp, vp, sz, dp]),
        "rk4_chain_integrate": (c_int, [H, vp, vp, vp, sz, i64, dp]),
        "rk4_chain_integrate_host": (c_int, [H, vp, vp, vp, vp, vp, sz, i64, dp]),
        "rk4_chain_energy": (c_int, [H, vp, vp, vp, sz, dp]),
        "rk4_chain_energy_static": (c_int, [H, vp, vp, dp]),
        "rk4_chain_status": (c_int, [H, vp]),
        "rk4_chain_set_option": (c_int, [H, c_int, i64]),
        "rk4_debug_barrier_timeout": (c_int, [H, vp, vp, vp, sz, i64]),
        "rk4_chain_set_time": (c_int, [H, ctypes.c_double]),
        "rk4_chain_get_clock": (c_int, [H, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]),
        "rk4_chain_set_clock": (c_int, [H, ctypes.c_double, i64]),
        "rk4_chain_set_tableau": (c_int, [H, c_int, dp, dp]),
        "rk4_chain_set_coupling2": (c_int, [H, ctypes.c_double]),
        "rk4_chain_set_site_params": (c_int, [H, vp]),
        "rk4_chain_destroy": (c_int, [H]),
        "rk4_strerror": (ctypes.c_char_p, [c_int]),
        "rk4_fill_uniform": (c_int, [vp, i64, ctypes.c_uint64, ctypes.c_uint64, c_int, vp]),
        "rk4_domain_create": (c_int, [ctypes.POINTER(H), c_int, c_int, i64, ctypes.c_double, c_int,
                                      ctypes.POINTER(rk4_params), c_int, ctypes.POINTER(i64), i64, vp]),
        "rk4_domain_part": (c_int, [H, c_int] + [ctypes.POINTER(i64)] * 5),
        "rk4_domain_shape": (c_int, [H, ctypes.POINTER(i64), ctypes.POINTER(c_int)]),
        "rk4_domain_chain": (c_int, [H, ctypes.POINTER(H)]),
        "rk4_domain_workspace_bytes": (c_int, [H, ctypes.POINTER(sz)]),
        "rk4_domain_scatter": (c_int, [H, vp, vp, vp, vp]),
        "rk4_domain_gather": (c_int, [H, vp, vp, vp, vp]),
        "rk4_domain_exchange": (c_int, [H, vp, vp]),
        "rk4_domain_integrate": (c_int, [H, vp, vp, vp, sz, i64, dp]),
        "rk4_domain_energy": (c_int, [H, vp, vp, vp, sz, dp]),
        "rk4_domain_status": (c_int, [H, vp]),
        "rk4_domain_destroy": (c_int, [H]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
_nchains_of: dict[int, int] = {}


def _nchains(h) -> int:
    return _nchains_of.get(h.value, 1)


def header_functions() -> list[str]:
    """Names of every function include/rk4chain.h declares."""
    text = open(HEADER_PATH).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rk4_[a-z0-9_]+)\s*\(", text)))


def _check(code: int, what: str):
    if code != RK4_OK:
        raise RK4Error(code, what)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)!r}")


def _nbytes(x) -> int:
    if hasattr(x, "element_size"):
        return x.numel() * x.element_size()
    if isinstance(x, np.ndarray):
        return x.nbytes
    raise TypeError("pass ws_bytes explicitly for raw pointers")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def _params(params):
    if params is None:
        p = rk4_params()
        _lib.rk4_params_default(ctypes.byref(p))
        return p
    if isinstance(params, rk4_params):
        return params
    p = rk4_params()
    _lib.rk4_params_default(ctypes.byref(p))
    for k, v in dict(params).items():
        setattr(p, k, float(v))
    return p


def rk4_strerror(code: int) -> str:
    return _lib.rk4_strerror(int(code)).decode()


def rk4_params_default() -> rk4_params:
    return _params(None)


def rk4_chain_create(model: int, precision: int, n: int, dt: float, bc: int, params=None, stream=None):
    h = ctypes.c_void_p()
    p = _params(params)
    _check(_lib.rk4_chain_create(ctypes.byref(h), int(model), int(precision), int(n), float(dt), int(bc),
                                 ctypes.byref(p), _stream(stream)), "rk4_chain_create")
    return h


def rk4_batch_create(model: int, precision: int, lengths, kappa, bc, dt: float, params=None, stream=None):
    lengths = np.ascontiguousarray(lengths, dtype=np.int64)
    kappa = np.ascontiguousarray(kappa, dtype=np.float64)
    bc = np.ascontiguousarray(bc, dtype=np.int8)
    if not (lengths.shape == kappa.shape == bc.shape) or lengths.ndim != 1:
        raise ValueError("lengths, kappa and bc must be 1-D arrays of one length")
    h = ctypes.c_void_p()
    p = _params(params)
    _check(_lib.rk4_batch_create(ctypes.byref(h), int(model), int(precision), int(lengths.shape[0]),
                                 lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 kappa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), float(dt), ctypes.byref(p),
                                 _stream(stream)), "rk4_batch_create")
    _nchains_of[h.value] = int(lengths.shape[0])  # rk4_chain_energy returns one value per chain
    return h


def rk4_chain_workspace_bytes(h) -> int:
    b = ctypes.c_size_t()
    _check(_lib.rk4_chain_workspace_bytes(h, ctypes.byref(b)), "rk4_chain_workspace_bytes")
    return int(b.value)


def rk4_chain_shape(h):
    n = ctypes.c_int64()
    d = ctypes.c_int()
    _check(_lib.rk4_chain_shape(h, ctypes.byref(n), ctypes.byref(d)), "rk4_chain_shape")
    return int(n.value), int(d.value)


def rk4_chain_set_kernel(h, kernel: int):
    _check(_lib.rk4_chain_set_kernel(h, int(kernel)), "rk4_chain_set_kernel")


def rk4_chain_set_tiling(h, block: int, v: int = 0, k: int = 0):
    _check(_lib.rk4_chain_set_tiling(h, int(block), int(v), int(k)), "rk4_chain_set_tiling")


def _tiling_dict(t: rk4_tiling) -> dict:
    return {"block": t.block, "v": t.v, "k": t.k, "G": t.G}


def rk4_chain_get_tiling(h) -> dict:
    t = rk4_tiling()
    _check(_lib.rk4_chain_get_tiling(h, ctypes.byref(t)), "rk4_chain_get_tiling")
    return _tiling_dict(t)


def rk4_chain_get_kernel(h) -> int:
    k = ctypes.c_int()
    _check(_lib.rk4_chain_get_kernel(h, ctypes.byref(k)), "rk4_chain_get_kernel")
    return int(k.value)


def rk4_chain_autotune(h, state, comp, ws, probe_steps: int = 16, ws_bytes: int | None = None) -> dict:
    t = rk4_tiling()
    wb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(_lib.rk4_chain_autotune(h, _ptr(state), _ptr(comp), _ptr(ws), wb, int(probe_steps), ctypes.byref(t)),
           "rk4_chain_autotune")
    return _tiling_dict(t)


def rk4_chain_step(h, state, comp, ws, ws_bytes: int | None = None) -> float:
    t = ctypes.c_double()
    wb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(_lib.rk4_chain_step(h, _ptr(state), _ptr(comp), _ptr(ws), wb, ctypes.byref(t)), "rk4_chain_step")
    return t.value


def rk4_chain_integrate(h, state, comp, ws, nsteps: int, ws_bytes: int | None = None) -> float:
    t = ctypes.c_double()
    wb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(_lib.rk4_chain_integrate(h, _ptr(state), _ptr(comp), _ptr(ws), wb, int(nsteps), ctypes.byref(t)),
           "rk4_chain_integrate")
    return t.value


def rk4_chain_integrate_host(h, host_state, host_comp, dev_state, dev_comp, ws, nsteps: int,
                             ws_bytes: int | None = None) -> float:
    t = ctypes.c_double()
    wb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(_lib.rk4_chain_integrate_host(h, _ptr(host_state), _ptr(host_comp), _ptr(dev_state), _ptr(dev_comp),
                                         _ptr(ws), wb, int(nsteps), ctypes.byref(t)), "rk4_chain_integrate_host")
    return t.value


def rk4_chain_energy(h, state, comp, ws, ws_bytes: int | None = None) -> np.ndarray:
    """FP64 energy (harmonic) or (1/2) sum |r|^2 (Roessler): one value per chain."""
    nchains = _nchains(h)
    out = np.zeros(max(nchains, 1), dtype=np.float64)
    wb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(_lib.rk4_chain_energy(h, _ptr(state), _ptr(comp), _ptr(ws), wb,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "rk4_chain_energy")
    return out


def rk4_chain_energy_static(h, state, comp) -> np.ndarray:
    """rk4_chain_energy without a workspace (scratch compiled into the library; for callers
    that cannot allocate device memory).  One value per chain."""
    out = np.zeros(max(_nchains(h), 1), dtype=np.float64)
    _check(_lib.rk4_chain_energy_static(h, _ptr(state), _ptr(comp), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "rk4_chain_energy_static")
    return out


def rk4_chain_status(h, ws) -> int:
    """The latched device status as an RK4_* code (does not raise)."""
    return int(_lib.rk4_chain_status(h, _ptr(ws)))


def rk4_chain_set_option(h, option: int, value: int):
    _check(_lib.rk4_chain_set_option(h, int(option), int(value)), "rk4_chain_set_option")


def rk4_debug_barrier_timeout(h, state, comp, ws, timeout_ns: int, ws_bytes: int | None = None):
    wb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(_lib.rk4_debug_barrier_timeout(h, _ptr(state), _ptr(comp), _ptr(ws), wb, int(timeout_ns)),
           "rk4_debug_barrier_timeout")


def rk4_chain_set_tableau(h, A=None, b=None):
    """Any explicit tableau (A strictly lower s x s, weights b, s <= 7); None restores RK4."""
    if A is None:
        _check(_lib.rk4_chain_set_tableau(h, 0, None, None), "rk4_chain_set_tableau")
        return
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    s = b.shape[0]
    if A.shape != (s, s):
        raise ValueError("tableau shape mismatch")
    dp = ctypes.POINTER(ctypes.c_double)
    _check(_lib.rk4_chain_set_tableau(h, s, A.ctypes.data_as(dp), b.ctypes.data_as(dp)), "rk4_chain_set_tableau")


def rk4_chain_set_coupling2(h, kappa2: float):
    _check(_lib.rk4_chain_set_coupling2(h, float(kappa2)), "rk4_chain_set_coupling2")


def rk4_chain_set_site_params(h, params):
    """Per-site parameters of a heterogeneous chain: a device tensor [total_sites, P] in the
    state's precision (P = 4 Roessler a, b, c, kappa; P = 2 harmonic omega^2, kappa), or None."""
    _check(_lib.rk4_chain_set_site_params(h, _ptr(params)), "rk4_chain_set_site_params")


def rk4_chain_get_clock(h):
    """(t0, steps taken): the handle's time is t0 + steps * dt."""
    t0 = ctypes.c_double()
    n = ctypes.c_int64()
    _check(_lib.rk4_chain_get_clock(h, ctypes.byref(t0), ctypes.byref(n)), "rk4_chain_get_clock")
    return t0.value, int(n.value)


def rk4_chain_set_clock(h, t0: float, nstep: int):
    _check(_lib.rk4_chain_set_clock(h, float(t0), int(nstep)), "rk4_chain_set_clock")


def rk4_chain_set_time(h, t0: float):
    _check(_lib.rk4_chain_set_time(h, float(t0)), "rk4_chain_set_time")


def rk4_chain_destroy(h):
    _nchains_of.pop(h.value, None)
    _check(_lib.rk4_chain_destroy(h), "rk4_chain_destroy")


def rk4_fill_uniform(dst, count: int, seed: int, start: int = 0, precision: int = RK4_FP64, stream=None):
    _check(_lib.rk4_fill_uniform(_ptr(dst), int(count), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                 int(start) & 0xFFFFFFFFFFFFFFFF, int(precision), _stream(stream)),
           "rk4_fill_uniform")


def rk4_domain_create(model: int, precision: int, n: int, dt: float, bc: int, nparts: int, ghost: int,
                      part_lengths=None, params=None, stream=None):
    """One chain split into `nparts` parts with `ghost` sites of ghost zone per side (see
    rk4_domain_part for the layout); part_lengths None splits evenly."""
    h = ctypes.c_void_p()
    p = _params(params)
    pl = None
    if part_lengths is not None:
        arr = np.ascontiguousarray(part_lengths, dtype=np.int64)
        if arr.shape != (int(nparts),):
            raise ValueError("part_lengths needs one entry per part")
        pl = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    _check(_lib.rk4_domain_create(ctypes.byref(h), int(model), int(precision), int(n), float(dt), int(bc),
                                  ctypes.byref(p), int(nparts), pl, int(ghost), _stream(stream)), "rk4_domain_create")
    return h


def rk4_domain_part(d, part: int) -> dict:
    v = [ctypes.c_int64() for _ in range(5)]
    _check(_lib.rk4_domain_part(d, int(part), *[ctypes.byref(x) for x in v]), "rk4_domain_part")
    return dict(zip(("first_site", "sites", "row", "ghost_left", "ghost_right"), (int(x.value) for x in v)))


def rk4_domain_shape(d):
    rows = ctypes.c_int64()
    dim = ctypes.c_int()
    _check(_lib.rk4_domain_shape(d, ctypes.byref(rows), ctypes.byref(dim)), "rk4_domain_shape")
    return int(rows.value), int(dim.value)


def rk4_domain_chain(d):
    """The batch handle that integrates the parts (owned by the domain: never destroy it)."""
    h = ctypes.c_void_p()
    _check(_lib.rk4_domain_chain(d, ctypes.byref(h)), "rk4_domain_chain")
    return h


def rk4_domain_workspace_bytes(d) -> int:
    b = ctypes.c_size_t()
    _check(_lib.rk4_domain_workspace_bytes(d, ctypes.byref(b)), "rk4_domain_workspace_bytes")
    return int(b.value)


def rk4_domain_scatter(d, chain_state, chain_comp, state, comp):
    _check(_lib.rk4_domain_scatter(d, _ptr(chain_state), _ptr(chain_comp), _ptr(state), _ptr(comp)),
           "rk4_domain_scatter")


def rk4_domain_gather(d, state, comp, chain_state, chain_comp):
    _check(_lib.rk4_domain_gather(d, _ptr(state), _ptr(comp), _ptr(chain_state), _ptr(chain_comp)),
           "rk4_domain_gather")


def rk4_domain_exchange(d, state, comp):
    _check(_lib.rk4_domain_exchange(d, _ptr(state), _ptr(comp)), "rk4_domain_exchange")


def rk4_domain_integrate(d, state, comp, ws, nsteps: int, ws_bytes: int | None = None) -> float:
    t = ctypes.c_double()
    wb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(_lib.rk4_domain_integrate(d, _ptr(state), _ptr(comp), _ptr(ws), wb, int(nsteps), ctypes.byref(t)),
           "rk4_domain_integrate")
    return t.value


def rk4_domain_energy(d, state, comp, ws, ws_bytes: int | None = None) -> float:
    out = ctypes.c_double()
    wb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(_lib.rk4_domain_energy(d, _ptr(state), _ptr(comp), _ptr(ws), wb, ctypes.byref(out)), "rk4_domain_energy")
    return out.value


def rk4_domain_status(d, ws) -> int:
    return int(_lib.rk4_domain_status(d, _ptr(ws)))


def rk4_domain_destroy(d):
    _check(_lib.rk4_domain_destroy(d), "rk4_domain_destroy")


from .chain import Chain  # noqa: E402  (convenience wrapper over the functions above)

__all__ = [n for n in dir() if n.startswith("rk4_") or n.startswith("RK4") or n in ("Chain",)]
