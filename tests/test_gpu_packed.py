"""Batches with packed tiles (Sec. 2.3's clusters applied to many chains at once).

A batch's chains are cut into full tiles of G interior sites; each chain's remaining piece (the
whole chain when it is shorter than G) is placed, with its own halo of 4k sites per side, next
to other chains' pieces in a shared tile.  Whatever the packing, every site performs the same
operations as in the one-stage-per-launch kernel, so the results must be bit-identical to it,
for chain lengths around every tile boundary, fixed and periodic ends, both precisions, every
number of sites per thread and both tiled schemes; and the staged result matches the oracle.
"""
import numpy as np
import pytest

import chain_inputs as ci
import closed_form as cf
import oracle
from tolerances import FP32_KAHAN_TOL

pytestmark = pytest.mark.gpu

# (block, v, k): tile width W = block v, G = W - 8k interior sites per full tile
TILINGS = [(256, 4, 1), (128, 4, 4), (256, 8, 8), (64, 4, 2), (1024, 1, 2), (128, 2, 4), (512, 2, 16)]


@pytest.fixture(scope="module")
def rk():
    import torch
    import paper_1412_0544_gb300 as m
    assert torch.cuda.is_available()
    return m


@pytest.fixture(scope="module")
def gh(rk):
    import gpu_helpers
    return gpu_helpers


def awkward_lengths():
    """Chain lengths around the tile boundaries of every tiling above (n = G - 1, G, G + 1,
    2G, 2G + 1), tiny chains (1, 2, 3 sites: a periodic chain shorter than its halo wraps
    many times) and a log-uniform spread."""
    L = {1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 33, 63, 64, 65, 127, 129}
    for b, v, k in TILINGS:
        G = b * v - 8 * k
        L.update({G - 1, G, G + 1, 2 * G, 2 * G + 1, 3 * G - 1})
    lengths = np.array(sorted(L), dtype=np.int64)
    extra, _, _ = ci.batch_spec(40, seed=600, nmin=1, nmax=5000)
    lengths = np.concatenate([lengths, extra])
    n = lengths.size
    kappa = 0.5 + 1.5 * ci.uniform01(601, 2, 0, n)
    bcs = (np.arange(n) % 2).astype(np.int8)  # alternate periodic and fixed ends
    return lengths, kappa, bcs


@pytest.mark.parametrize("precision", [0, 1])
def test_packed_batch_bitwise_equals_staged(rk, gh, precision):
    lengths, kappa, bcs = awkward_lengths()
    fp32 = precision == rk.RK4_FP32_KAHAN
    y0 = ci.uniform_state(int(lengths.sum()), 3, seed=602)
    if fp32:
        y0 = y0.astype(np.float32)
    T = 37
    st, cst = gh.gpu_run(y0, precision=precision, nsteps=T, lengths=lengths, kappas=kappa, bcs=bcs,
                         kernel=rk.RK4_KERNEL_STAGED, return_comp=True)
    for kernel in (rk.RK4_KERNEL_BLOCKED, rk.RK4_KERNEL_PERSISTENT):
        for tiling in TILINGS:
            got, cgot = gh.gpu_run(y0, precision=precision, nsteps=T, lengths=lengths, kappas=kappa, bcs=bcs,
                                   kernel=kernel, tiling=tiling, return_comp=True)
            assert np.array_equal(got, st), (kernel, tiling)
            if fp32:
                assert np.array_equal(cgot, cst), (kernel, tiling)
    ref = oracle.batch_rk4_integrate(y0.astype(np.float64), lengths, kappa, bcs, nsteps=T)
    err = cf.rel_inf(st - (cst if fp32 else 0.0), ref)
    assert err <= (1e-12 if not fp32 else FP32_KAHAN_TOL), err


def test_packed_batch_many_tiny_chains(rk, gh):
    """Thousands of chains of 1..40 sites: dozens of segments share each tile."""
    lengths, kappa, bcs = ci.batch_spec(3000, seed=610, nmin=1, nmax=40)
    y0 = ci.uniform_state(int(lengths.sum()), 3, seed=611)
    st = gh.gpu_run(y0, nsteps=24, lengths=lengths, kappas=kappa, bcs=bcs, kernel=rk.RK4_KERNEL_STAGED)
    for kernel in (rk.RK4_KERNEL_BLOCKED, rk.RK4_KERNEL_PERSISTENT):
        for tiling in [(256, 4, 2), (512, 2, 1), (256, 8, 6)]:
            got = gh.gpu_run(y0, nsteps=24, lengths=lengths, kappas=kappa, bcs=bcs, kernel=kernel, tiling=tiling)
            assert np.array_equal(got, st), (kernel, tiling)
    ref = oracle.batch_rk4_integrate(y0, lengths, kappa, bcs, nsteps=24)
    assert cf.rel_inf(st, ref) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_without_tile_table_bitwise_equals_staged(rk, gh, precision):
    """A tile finds its chain in a table of the launch's full tiles, which the workspace holds for
    tiles of at least 64 interior sites.  At 64 x 2 x 8 (W = 128, halo 32 per side, G = 61 in
    FP32 and 63 in FP64 after the 16-byte window alignment) these long chains have more full
    tiles than the table holds, so the launches search the first-tile prefix instead; both ways
    must give the staged kernel's result bit for bit."""
    fp32 = precision == rk.RK4_FP32_KAHAN
    lengths = np.array([100000, 70001, 5, 3000, 1], dtype=np.int64)
    G = 61 if fp32 else 63
    assert sum(n // G for n in lengths) > lengths.sum() // 64 + lengths.size  # beyond the table
    kappa = np.array([1.0, 0.7, 1.3, 0.9, 1.1])
    bcs = np.array([0, 1, 0, 1, 0], dtype=np.int8)
    y0 = ci.uniform_state(int(lengths.sum()), 3, seed=620)
    if fp32:
        y0 = y0.astype(np.float32)
    T = 21
    st, cst = gh.gpu_run(y0, precision=precision, nsteps=T, lengths=lengths, kappas=kappa, bcs=bcs,
                         kernel=rk.RK4_KERNEL_STAGED, return_comp=True)
    for kernel in (rk.RK4_KERNEL_BLOCKED, rk.RK4_KERNEL_PERSISTENT):
        for tiling in [(64, 2, 8), (256, 4, 2)]:  # without and with the table
            got, cgot = gh.gpu_run(y0, precision=precision, nsteps=T, lengths=lengths, kappas=kappa, bcs=bcs,
                                   kernel=kernel, tiling=tiling, return_comp=True)
            assert np.array_equal(got, st), (kernel, tiling)
            if fp32:
                assert np.array_equal(cgot, cst), (kernel, tiling)
