"""Canary guard bands around every device buffer the library touches (state, compensation,
per-site parameters, workspace): each buffer is a view into a larger allocation whose margins
hold a bit pattern; after integrations and reductions through every scheme, the margins must be
unchanged.  A write outside a buffer's extent (an indexing slip at a ragged tile, a chain end, a
wrap) would show up here.  Sizes are ragged on purpose."""
import numpy as np
import pytest

import chain_inputs as ci
import oracle_pins as P

pytestmark = pytest.mark.gpu

GUARD = 4096  # bytes of margin on each side of every buffer
PATTERN = 0xA5


@pytest.fixture(scope="module")
def rk():
    import torch
    import paper_1412_0544_gb300 as m
    assert torch.cuda.is_available()
    return m


class Guarded:
    """A device buffer of `nbytes` with canary margins (the buffer itself stays 256-B aligned)."""

    def __init__(self, nbytes):
        import torch
        self.nbytes = nbytes
        self.raw = torch.full((GUARD + nbytes + GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
        self.view = self.raw[GUARD:GUARD + nbytes]

    def typed(self, dtype, shape):
        return self.view.view(dtype).view(*shape)

    def intact(self):
        r = self.raw.cpu().numpy()
        return bool(np.all(r[:GUARD] == PATTERN) and np.all(r[GUARD + self.nbytes:] == PATTERN))


def run_guarded(rk, y0, *, model=0, prec=0, bc=0, kernel=0, tiling=None, nsteps=9, lengths=None, kappas=None,
                bcs=None, sp=None, tableau=None, kappa2=0.0):
    import torch
    dtype = torch.float32 if prec else torch.float64
    es = 4 if prec else 8
    n, D = y0.shape
    if lengths is not None:
        h = rk.rk4_batch_create(model, prec, lengths, kappas, bcs, 0.01)
    else:
        h = rk.rk4_chain_create(model, prec, n, 0.01, bc)
    bufs = []
    try:
        if tableau is not None:
            rk.rk4_chain_set_tableau(h, *tableau)
        if kappa2:
            rk.rk4_chain_set_coupling2(h, kappa2)
        if sp is not None:
            g = Guarded(sp.size * es)
            g.typed(dtype, sp.shape).copy_(torch.from_numpy(sp).to(dtype))
            rk.rk4_chain_set_site_params(h, g.view)
            bufs.append(g)
        rk.rk4_chain_set_kernel(h, kernel)
        if tiling is not None:
            rk.rk4_chain_set_tiling(h, *tiling)
        gs = Guarded(n * D * es)
        st = gs.typed(dtype, (n, D))
        st.copy_(torch.from_numpy(y0).to(dtype))
        bufs.append(gs)
        cp = None
        if prec:
            gc = Guarded(n * D * es)
            cp = gc.typed(dtype, (n, D))
            cp.zero_()
            bufs.append(gc)
        wsb = rk.rk4_chain_workspace_bytes(h)
        gw = Guarded(wsb)
        bufs.append(gw)
        rk.rk4_chain_integrate(h, st, cp, gw.view, nsteps, ws_bytes=wsb)
        if model == 0 or sp is None:
            rk.rk4_chain_energy(h, st, cp, gw.view, ws_bytes=wsb)
        torch.cuda.synchronize()
        return all(b.intact() for b in bufs)
    finally:
        rk.rk4_chain_destroy(h)


CASES = [
    dict(kernel=1), dict(kernel=2, tiling=(64, 1, 1)), dict(kernel=2, tiling=(256, 4, 4)),
    dict(kernel=2, tiling=(128, 8, 16)), dict(kernel=3, tiling=(128, 4, 2)),
]


@pytest.mark.parametrize("case", CASES, ids=[str(c) for c in CASES])
@pytest.mark.parametrize("prec,bc,n", [(0, 0, 1), (0, 1, 3), (1, 0, 777), (0, 1, 10001), (1, 1, 4099)])
def test_single_chain_guards(rk, case, prec, bc, n):
    y0 = ci.uniform_state(n, 3, seed=500 + n)
    assert run_guarded(rk, y0, prec=prec, bc=bc, **case)


@pytest.mark.parametrize("kernel", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_batch_guards(rk, kernel, prec):
    lengths, kappa, bcs = ci.batch_spec(37, seed=510, nmin=1, nmax=900)
    y0 = ci.uniform_state(int(lengths.sum()), 3, seed=511)
    assert run_guarded(rk, y0, prec=prec, kernel=kernel, tiling=(128, 4, 4), lengths=lengths, kappas=kappa, bcs=bcs)


@pytest.mark.parametrize("kernel", [1, 2])
def test_generic_and_heterogeneous_guards(rk, kernel):
    A, b, _ = P.TABLEAUX["dopri5"]
    y0 = ci.uniform_state(3331, 3, seed=520)
    assert run_guarded(rk, y0, bc=1, kernel=kernel, tableau=(A, b), kappa2=0.4,
                       tiling=(128, 4, 2) if kernel == 2 else None)
    sp = P.het_params(3331, 0, 521)
    assert run_guarded(rk, y0, prec=1, bc=0, kernel=kernel, sp=sp, tiling=(256, 2, 4) if kernel == 2 else None)
