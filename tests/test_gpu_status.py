"""The status word reports a blow-up: with a step far outside RK4's stability region the state
overflows to infinity and NaN, every scheme that stores such values latches RK4_ENONFINITE,
and rk4_chain_status returns it (no reduction needed); a stable run reports RK4_OK.  Overflow
is ordinary floating-point arithmetic on the GPU, not a fault."""
import numpy as np
import pytest

import chain_inputs as ci
import oracle_pins as P

pytestmark = pytest.mark.gpu

PER, FIX = 0, 1
ROE, HAR = 0, 1


@pytest.fixture(scope="module")
def rk():
    import torch
    import paper_1412_0544_gb300 as m
    assert torch.cuda.is_available()
    return m


def run_status(rk, model, prec, dt, nsteps, *, n=5003, bc=PER, kernel=None, tiling=None, batch=False,
               tableau=None, site_params=False):
    import torch
    D = 3 if model == ROE else 2
    dtype = torch.float32 if prec else torch.float64
    if batch:
        lengths, kappa, bcs = ci.batch_spec(40, seed=900, nmin=1, nmax=400)
        n = int(lengths.sum())
        h = rk.rk4_batch_create(model, prec, lengths, kappa, bcs, dt)
    else:
        h = rk.rk4_chain_create(model, prec, n, dt, bc)
    try:
        if kernel is not None:
            rk.rk4_chain_set_kernel(h, kernel)
        if tableau is not None:
            rk.rk4_chain_set_tableau(h, *tableau)
        sp = None
        if site_params:
            sp = torch.from_numpy(P.het_params(n, model, 901)).to(dtype).cuda()
            rk.rk4_chain_set_site_params(h, sp)
        if tiling is not None:
            rk.rk4_chain_set_tiling(h, *tiling)
        st = torch.from_numpy(ci.uniform_state(n, D, seed=902)).to(dtype).cuda()
        cp = torch.zeros_like(st) if prec else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
        code = rk.rk4_chain_status(h, ws)
        finite = bool(torch.isfinite(st).all())
        return code, finite
    finally:
        rk.rk4_chain_destroy(h)


SCHEMES = [
    dict(kernel=1), dict(kernel=2, tiling=(256, 4, 1)), dict(kernel=2, tiling=(128, 8, 16)), dict(batch=True),
    dict(batch=True, kernel=2, tiling=(128, 4, 4)), dict(kernel=2, tableau="dopri5"), dict(kernel=1, tableau="dopri5"),
    dict(kernel=2, site_params=True, tiling=(256, 2, 4)), dict(kernel=2, bc=FIX, tiling=(256, 4, 2)),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("scheme", SCHEMES, ids=[str(s) for s in SCHEMES])
def test_blow_up_is_reported(rk, prec, scheme):
    kw = dict(scheme)
    if kw.get("tableau") == "dopri5":
        A, b, _ = P.TABLEAUX["dopri5"]
        kw["tableau"] = (A, b)
    # harmonic chain, dt = 5: |R(i w dt)| ~ 650 per step, overflow well within 300 steps
    code, finite = run_status(rk, HAR, prec, 5.0, 300, **kw)
    assert not finite
    assert code == rk.RK4_ENONFINITE
    code, finite = run_status(rk, HAR, prec, 0.01, 30, **kw)
    assert finite and code == rk.RK4_OK


def test_status_is_cleared_by_the_next_integration(rk):
    import torch
    h = rk.rk4_chain_create(HAR, 0, 3001, 5.0, PER)
    try:
        st = torch.from_numpy(ci.uniform_state(3001, 2, seed=903)).cuda()
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_integrate(h, st, None, ws, 300)
        torch.cuda.synchronize()
        st.copy_(torch.from_numpy(ci.uniform_state(3001, 2, seed=904)))
        rk.rk4_chain_integrate(h, st, None, ws, 1)  # one unstable step stays finite
        assert bool(torch.isfinite(st).all())
        assert rk.rk4_chain_status(h, ws) == rk.RK4_OK
    finally:
        rk.rk4_chain_destroy(h)
