"""Serial FP64 CPU oracle for RK integration of nearest-neighbour chains.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The CUDA library never calls it and shares no
code with it.

The arithmetic lives in ``rk4_oracle.c`` (plain C, compiled with ``-ffp-contract=off``); this
module only compiles it with gcc and marshals numpy arrays.  What the C file computes, and the
paper passages it follows (Eqs. (2)-(7) of arXiv:1412.0544 and the classical RK4 tableau), is
stated in its header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

ROESSLER, HARMONIC = 0, 1
PERIODIC, FIXED = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rk4_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librk4oracle.so")
_lock = threading.Lock()
_lib = None

# Classical fourth-order tableau (Sec. 2 of the paper cites Press et al.): kept here only to
# hand general tableaux to the C routine; the default integrator uses the C copy.
RK4_A = np.array([[0, 0, 0, 0], [0.5, 0, 0, 0], [0, 0.5, 0, 0], [0, 0, 1.0, 0]], dtype=np.float64)
RK4_B = np.array([1 / 6, 1 / 3, 1 / 3, 1 / 6], dtype=np.float64)


def dim(model: int) -> int:
    return {ROESSLER: 3, HARMONIC: 2}[model]


def build(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile the oracle (gcc, serial, no FMA contraction) and return the .so path."""
    src = src or _SRC
    out = out or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-o", tmp, src, "-lm"],
            check=True,
        )
        os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load (building if needed) the oracle library; returns the ctypes handle."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    lib.oracle_rk_integrate.argtypes = [ctypes.c_int, ctypes.c_int, i64, dp, ctypes.c_int, dp, dp,
                                        ctypes.c_double, i64, dp]
    lib.oracle_rk_integrate.restype = ctypes.c_int
    lib.oracle_rk4_integrate.argtypes = [ctypes.c_int, ctypes.c_int, i64, dp, ctypes.c_double, i64, dp]
    lib.oracle_rk4_integrate.restype = ctypes.c_int
    lib.oracle_rhs.argtypes = [ctypes.c_int, ctypes.c_int, i64, dp, dp, dp]
    lib.oracle_rhs.restype = ctypes.c_int
    lib.oracle_rk4_integrate_het.argtypes = [ctypes.c_int, ctypes.c_int, i64, dp, ctypes.c_double, i64, dp]
    lib.oracle_rk4_integrate_het.restype = ctypes.c_int
    lib.oracle_energy_harmonic.argtypes = [ctypes.c_int, i64, dp, dp]
    lib.oracle_energy_harmonic.restype = ctypes.c_double
    lib.oracle_half_norm2.argtypes = [i64, dp]
    lib.oracle_half_norm2.restype = ctypes.c_double
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params(a=0.2, b=1.0, c=9.0, kappa=1.0, omega0=1.0, kappa2=0.0) -> np.ndarray:
    """Parameter vector (a, b, c, kappa, omega0, kappa2); defaults are Sec. 3.1's a=0.2, b=1,
    c=9 with nearest-neighbour coupling only (kappa2 = 0)."""
    return np.array([a, b, c, kappa, omega0, kappa2], dtype=np.float64)


def _state(y0, model) -> np.ndarray:
    y = np.array(y0, dtype=np.float64, copy=True, order="C")
    D = dim(model)
    if y.ndim == 1:
        y = y.reshape(-1, D)
    if y.ndim != 2 or y.shape[1] != D:
        raise ValueError(f"state must be [N, {D}]")
    return y


def rk4_integrate(y0, model=ROESSLER, bc=PERIODIC, dt=0.01, nsteps=1, prm=None, lib=None) -> np.ndarray:
    """Classical RK4 over nsteps; returns a new [N, D] float64 array."""
    lib = lib or load()
    y = _state(y0, model)
    prm = params() if prm is None else np.asarray(prm, dtype=np.float64)
    rc = lib.oracle_rk4_integrate(model, bc, y.shape[0], _dp(prm), float(dt), int(nsteps), _dp(y))
    if rc != 0:
        raise ValueError(f"oracle_rk4_integrate failed: {rc}")
    return y


def site_param_count(model: int) -> int:
    """Per-site parameters of a heterogeneous chain: Roessler a, b, c, kappa; harmonic omega^2, kappa."""
    return {ROESSLER: 4, HARMONIC: 2}[model]


def rk4_integrate_het(y0, site_params, model=ROESSLER, bc=PERIODIC, dt=0.01, nsteps=1, lib=None) -> np.ndarray:
    """Classical RK4 on a heterogeneous chain (Eq. (1)): site_params is [N, P]."""
    lib = lib or load()
    y = _state(y0, model)
    sp = np.ascontiguousarray(site_params, dtype=np.float64)
    if sp.shape != (y.shape[0], site_param_count(model)):
        raise ValueError("site_params must be [N, P]")
    rc = lib.oracle_rk4_integrate_het(model, bc, y.shape[0], _dp(sp), float(dt), int(nsteps), _dp(y))
    if rc != 0:
        raise ValueError(f"oracle_rk4_integrate_het failed: {rc}")
    return y


def rk_integrate(y0, A, b, model=ROESSLER, bc=PERIODIC, dt=0.01, nsteps=1, prm=None, lib=None) -> np.ndarray:
    """Any explicit tableau (A strictly lower s x s, weights b) over nsteps."""
    lib = lib or load()
    y = _state(y0, model)
    prm = params() if prm is None else np.asarray(prm, dtype=np.float64)
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    s = b.shape[0]
    if A.shape != (s, s):
        raise ValueError("tableau shape mismatch")
    rc = lib.oracle_rk_integrate(model, bc, y.shape[0], _dp(prm), s, _dp(A), _dp(b), float(dt), int(nsteps), _dp(y))
    if rc != 0:
        raise ValueError(f"oracle_rk_integrate failed: {rc}")
    return y


def rhs(r, model=ROESSLER, bc=PERIODIC, prm=None, lib=None) -> np.ndarray:
    lib = lib or load()
    r = _state(r, model)
    k = np.empty_like(r)
    prm = params() if prm is None else np.asarray(prm, dtype=np.float64)
    rc = lib.oracle_rhs(model, bc, r.shape[0], _dp(prm), _dp(r), _dp(k))
    if rc != 0:
        raise ValueError(f"oracle_rhs failed: {rc}")
    return k


def energy_harmonic(y, bc=PERIODIC, prm=None, lib=None) -> float:
    lib = lib or load()
    y = _state(y, HARMONIC)
    prm = params() if prm is None else np.asarray(prm, dtype=np.float64)
    return float(lib.oracle_energy_harmonic(bc, y.shape[0], _dp(prm), _dp(y)))


def half_norm2(y, lib=None) -> float:
    lib = lib or load()
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
    return float(lib.oracle_half_norm2(y.shape[0], _dp(y)))


def batch_rk4_integrate(y0_concat, lengths, kappas, bcs, model=ROESSLER, dt=0.01, nsteps=1, prm=None,
                        lib=None) -> np.ndarray:
    """Independent chains stored back to back; each has its own length, kappa and boundary."""
    lib = lib or load()
    y = _state(y0_concat, model)
    prm = params() if prm is None else np.asarray(prm, dtype=np.float64)
    off = 0
    for n, kap, bc in zip(lengths, kappas, bcs):
        n = int(n)
        p = prm.copy()
        p[3] = float(kap)
        seg = np.ascontiguousarray(y[off:off + n])
        rc = lib.oracle_rk4_integrate(model, int(bc), n, _dp(p), float(dt), int(nsteps), _dp(seg))
        if rc != 0:
            raise ValueError(f"oracle_rk4_integrate failed: {rc}")
        y[off:off + n] = seg
        off += n
    if off != y.shape[0]:
        raise ValueError("lengths do not sum to the state size")
    return y
