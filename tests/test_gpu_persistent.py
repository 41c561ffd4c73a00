"""The persistent cooperative kernel on awkward tile shapes: state and compensation must equal
the one-stage-per-launch kernel bit for bit for chains whose last tile is shorter than the
halo (that tile's window wraps past the first tile), chains shorter than one tile, uneven
batches whose plan ends with tail time blocks of other k, many time blocks and many small
tiles, over repeated runs (items are handed out dynamically, so the block-to-tile mapping
differs from run to run)."""
import numpy as np
import pytest

import chain_inputs as ci

pytestmark = pytest.mark.gpu

PER, FIX = 0, 1
ROE, HAR = 0, 1


@pytest.fixture(scope="module")
def rk():
    import torch
    import paper_1412_0544_gb300 as m
    assert torch.cuda.is_available()
    return m


def run(rk, y0, *, prec, nsteps, kernel, tiling=None, bc=PER, model=ROE, batch=None):
    import torch
    if batch is not None:
        lengths, kappa, bcs = batch
        h = rk.rk4_batch_create(model, prec, lengths, kappa, bcs, 0.01)
    else:
        h = rk.rk4_chain_create(model, prec, y0.shape[0], 0.01, bc)
    try:
        rk.rk4_chain_set_kernel(h, kernel)
        if tiling is not None:
            rk.rk4_chain_set_tiling(h, *tiling)
        dtype = torch.float32 if prec else torch.float64
        st = torch.from_numpy(np.ascontiguousarray(y0)).to(dtype).cuda()
        cp = torch.zeros_like(st) if prec else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
        code = rk.rk4_chain_status(h, ws)
        assert code == rk.RK4_OK, code
        out = st.cpu().numpy()
        return (out, cp.cpu().numpy()) if prec else (out, None)
    finally:
        rk.rk4_chain_destroy(h)


def same(a, b):
    return np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8)) and (
        a[1] is None or np.array_equal(a[1].view(np.uint8), b[1].view(np.uint8)))


# tiling (128, 4, 8): W = 512, H = 32, G = 448; n = 10 G + 5 leaves a 5-site last tile
CASES = [
    dict(n=10 * 448 + 5, bc=PER, tiling=(128, 4, 8)),
    dict(n=10 * 448 + 5, bc=FIX, tiling=(128, 4, 8)),
    dict(n=448 + 31, bc=PER, tiling=(128, 4, 8)),   # two tiles, the second shorter than H
    dict(n=300, bc=PER, tiling=(128, 4, 8)),        # shorter than one tile
    dict(n=70001, bc=PER, tiling=(256, 4, 2)),
    dict(n=33333, bc=FIX, tiling=(128, 8, 4)),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[f"n{c['n']}_bc{c['bc']}_{c['tiling']}" for c in CASES])
def test_persistent_bitwise(rk, prec, case):
    D = 3
    y0 = ci.uniform_state(case["n"], D, seed=990 + case["n"] % 97)
    if prec:
        y0 = y0.astype(np.float32)
    nsteps = 37 * case["tiling"][2]  # 37 time blocks (36 of k and two of k / 2)
    ref = run(rk, y0, prec=prec, nsteps=nsteps, kernel=rk.RK4_KERNEL_STAGED, bc=case["bc"])
    for _ in range(3):
        got = run(rk, y0, prec=prec, nsteps=nsteps, kernel=rk.RK4_KERNEL_PERSISTENT, tiling=case["tiling"],
                  bc=case["bc"])
        assert same(got, ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_persistent_batch_with_tails(rk, prec):
    """Uneven chains (many shorter than a tile, many with short last tiles), a step count whose
    plan ends with a tail time block of another k."""
    lengths, kappa, bcs = ci.batch_spec(300, seed=991, nmin=1, nmax=5000)
    y0 = ci.uniform_state(int(lengths.sum()), 3, seed=992)
    if prec:
        y0 = y0.astype(np.float32)
    b = (lengths, kappa, bcs)
    nsteps = 5 * 8 + 5  # 5 time blocks at k = 8, then a tail of k = 5
    ref = run(rk, y0, prec=prec, nsteps=nsteps, kernel=rk.RK4_KERNEL_STAGED, batch=b)
    for _ in range(3):
        got = run(rk, y0, prec=prec, nsteps=nsteps, kernel=rk.RK4_KERNEL_PERSISTENT, tiling=(128, 4, 8), batch=b)
        assert same(got, ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_persistent_batch_many_tiles_per_block(rk, prec):
    """A batch large enough that every resident block draws several full tiles per time block
    (and the block order in which tiles are drawn differs from run to run): bit for bit the
    staged result, over repeated runs, with periodic and fixed chains, wrapped end windows,
    packed pieces and a tail time block of another k."""
    lengths, kappa, bcs = ci.batch_spec(72, seed=994, nmin=2000, nmax=90000)
    y0 = ci.uniform_state(int(lengths.sum()), 3, seed=995)
    if prec:
        y0 = y0.astype(np.float32)
    b = (lengths, kappa, bcs)
    nsteps = 4 * 4 + 2  # four time blocks of k = 4, then a tail of k = 2
    ref = run(rk, y0, prec=prec, nsteps=nsteps, kernel=rk.RK4_KERNEL_STAGED, batch=b)
    for tiling in [(128, 4, 4), (256, 4, 4), (64, 2, 4), (256, 8, 4)]:
        for _ in range(2):
            got = run(rk, y0, prec=prec, nsteps=nsteps, kernel=rk.RK4_KERNEL_PERSISTENT, tiling=tiling, batch=b)
            assert same(got, ref), tiling


def test_persistent_harmonic_many_small_tiles(rk):
    """128 x 1 tiles with k = 4 (G = 96): thousands of items per time block, 100 time blocks."""
    n = 200003
    y0 = ci.uniform_state(n, 2, seed=993)
    ref = run(rk, y0, prec=0, nsteps=400, kernel=rk.RK4_KERNEL_STAGED, model=HAR)
    got = run(rk, y0, prec=0, nsteps=400, kernel=rk.RK4_KERNEL_PERSISTENT, tiling=(128, 1, 4), model=HAR)
    assert same(got, ref)
