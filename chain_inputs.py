"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the benchmark.

This module draws random numbers and nothing else: it holds none of the integration
arithmetic.  Every value comes from the counter-based SplitMix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the value with counter
j under key s is the first output of a SplitMix64 generator whose state is ``s XOR j``, i.e.

    z  = (s ^ j) + 0x9E3779B97F4A7C15        (mod 2^64)
    z  = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z  = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z ^= z >> 31

and a uniform double in [0, 1) is ``(z >> 11) * 2^-53``.  The CUDA library carries its own
implementation of the same published definition (for filling multi-gigabyte states on the
device); the tests check the two agree bit for bit.

Workload recipe (the paper starts from "random initial conditions", Sec. 3.2):
  * state component d of site i (global index j = i*D + d) is v = 2u - 1, u uniform[0,1)
    from stream 0, i.e. i.i.d. uniform[-1, 1); FP32 runs start from float(v), rounded to
    nearest;
  * batches of chains: lengths round(exp(U(ln 64, ln 65536))), coupling kappa ~ U[0.5, 2],
    boundary periodic/fixed with probability 1/2 each, from streams 1, 2 and 3.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 0x14120544
GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
STREAM_STATE, STREAM_LENGTH, STREAM_KAPPA, STREAM_BC = 0, 1, 2, 3


def _stream_key(seed: int, stream: int) -> np.uint64:
    # streams are separated in the top byte of the counter
    return np.uint64((int(seed) ^ (int(stream) << 56)) & 0xFFFFFFFFFFFFFFFF)


def splitmix64(keys: np.ndarray) -> np.ndarray:
    """First SplitMix64 output for each 64-bit state in ``keys`` (uint64 array)."""
    z = np.asarray(keys, dtype=np.uint64) + GOLDEN
    z = (z ^ (z >> np.uint64(30))) * M1
    z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Doubles (z >> 11) * 2^-53 for counters start .. start+count-1 of a stream."""
    j = np.arange(start, start + count, dtype=np.uint64)
    z = splitmix64(j ^ _stream_key(seed, stream))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_state(n: int, D: int, seed: int = DEFAULT_SEED, dtype=np.float64, chunk: int = 1 << 24) -> np.ndarray:
    """[n, D] state with i.i.d. uniform[-1, 1) components (exact in FP64, RN to FP32)."""
    total = int(n) * int(D)
    out = np.empty(total, dtype=dtype)
    for s in range(0, total, chunk):
        c = min(chunk, total - s)
        v = 2.0 * uniform01(seed, STREAM_STATE, s, c) - 1.0
        out[s:s + c] = v.astype(dtype)
    return out.reshape(int(n), int(D))


def batch_spec(nchains: int, seed: int = DEFAULT_SEED, nmin: int = 64, nmax: int = 65536):
    """Per-chain (lengths int64, kappa float64, bc int8) for a batch of uneven chains."""
    u_len = uniform01(seed, STREAM_LENGTH, 0, nchains)
    lengths = np.rint(np.exp(np.log(nmin) + u_len * (np.log(nmax) - np.log(nmin)))).astype(np.int64)
    lengths = np.clip(lengths, nmin, nmax)
    kappa = 0.5 + 1.5 * uniform01(seed, STREAM_KAPPA, 0, nchains)
    bc = (uniform01(seed, STREAM_BC, 0, nchains) < 0.5).astype(np.int8)  # 0 periodic, 1 fixed
    return lengths, kappa, bc
