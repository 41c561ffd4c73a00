"""GPU tests of the sub-domain decomposition (rk4_domain_*): one chain split into parts with
ghost zones, exchanged by device-to-device copies every floor(ghost / reach) steps, must give
the bits of the undivided chain (state and Kahan compensation) for every kernel scheme, model,
precision and boundary, ragged parts included; its energy must match the whole chain's up to
summation order."""
import numpy as np
import pytest

import chain_inputs as ci
import closed_form as cf
import oracle
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


def tensors(y0, prec):
    import torch
    dtype = torch.float32 if prec else torch.float64
    st = torch.from_numpy(np.ascontiguousarray(y0)).to(dtype).cuda()
    cp = torch.zeros_like(st) if prec else None
    return st, cp


def whole(rk, y0, model, prec, bc, nsteps, setup=None):
    import torch
    h = rk.rk4_chain_create(model, prec, y0.shape[0], 0.01, bc)
    try:
        if setup:
            setup(h)
        st, cp = tensors(y0, prec)
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
        e = rk.rk4_chain_energy(h, st, cp, ws)[0]
        torch.cuda.synchronize()
        return st.double().cpu().numpy(), (cp.double().cpu().numpy() if prec else None), e
    finally:
        rk.rk4_chain_destroy(h)


def domain(rk, y0, model, prec, bc, nparts, ghost, nsteps, lengths=None, setup=None, kernel=None, tiling=None):
    import torch
    n, D = y0.shape
    d = rk.rk4_domain_create(model, prec, n, 0.01, bc, nparts, ghost, part_lengths=lengths)
    try:
        h = rk.rk4_domain_chain(d)
        if setup:
            setup(h)
        if kernel is not None:
            rk.rk4_chain_set_kernel(h, kernel)
        if tiling is not None:
            rk.rk4_chain_set_tiling(h, *tiling)
        rows, dim = rk.rk4_domain_shape(d)
        assert dim == D
        cst, ccp = tensors(y0, prec)
        dtype = cst.dtype
        st = torch.full((rows, D), float("nan"), dtype=dtype, device="cuda")  # ghosts must be filled
        cp = torch.zeros_like(st) if prec else None
        ws = torch.empty(rk.rk4_domain_workspace_bytes(d), dtype=torch.uint8, device="cuda")
        rk.rk4_domain_scatter(d, cst, ccp, st, cp)
        t = rk.rk4_domain_integrate(d, st, cp, ws, nsteps)
        e = rk.rk4_domain_energy(d, st, cp, ws)
        out = torch.full_like(cst, float("nan"))
        oc = torch.full_like(cst, float("nan")) if prec else None
        rk.rk4_domain_gather(d, st, cp, out, oc)
        torch.cuda.synchronize()
        assert rk.rk4_domain_status(d, ws) == rk.RK4_OK
        assert t == pytest.approx(nsteps * 0.01, rel=1e-15)
        return out.double().cpu().numpy(), (oc.double().cpu().numpy() if prec else None), e
    finally:
        rk.rk4_domain_destroy(d)


N = 20011
CASES = [
    (ROE, 0, PER, 4, 8, None, 37),
    (ROE, 1, PER, 3, 16, [9000, 16, 10995], 50),
    (HAR, 0, FIX, 5, 12, None, 29),
    (HAR, 1, FIX, 2, 4, None, 10),
    (ROE, 0, PER, 1, 4, None, 13),
    (ROE, 1, FIX, 1, 0, None, 13),
    (ROE, 0, FIX, 7, 9, [3000, 9, 5000, 2002, 4000, 3000, 3000], 41),
    (HAR, 0, PER, 2, 5, None, 23),
]


@pytest.mark.parametrize("model,prec,bc,nparts,ghost,lengths,nsteps", CASES)
def test_domain_bitwise_vs_whole_chain(rk, model, prec, bc, nparts, ghost, lengths, nsteps):
    D = 3 if model == ROE else 2
    y0 = ci.uniform_state(N, D, seed=700 + nparts + 10 * model + 20 * prec)
    if prec:
        y0 = y0.astype(np.float32)
    ref, rc, re = whole(rk, y0, model, prec, bc, nsteps)
    got, gc, ge = domain(rk, y0, model, prec, bc, nparts, ghost, nsteps, lengths)
    assert np.array_equal(got, ref)
    if prec:
        assert np.array_equal(gc, rc)
    assert ge == pytest.approx(re, rel=1e-13)


def test_domain_vs_oracle(rk):
    y0 = ci.uniform_state(5003, 3, seed=710)
    ref = oracle.rk4_integrate(y0, ROE, PER, 0.01, 200)
    got, _, e = domain(rk, y0, ROE, 0, PER, 6, 20, 200)
    assert cf.rel_inf(got, ref) <= 1e-12
    assert e == pytest.approx(oracle.half_norm2(ref), rel=1e-13)


@pytest.mark.parametrize("kernel,tiling", [(1, None), (2, (128, 2, 1)), (2, (256, 4, 8)), (3, (128, 8, 4)),
                                           (3, (512, 2, 8))])
def test_domain_every_scheme(rk, kernel, tiling):
    y0 = ci.uniform_state(N, 3, seed=720).astype(np.float32)
    ref, rc, _ = whole(rk, y0, ROE, 1, PER, 33)
    got, gc, _ = domain(rk, y0, ROE, 1, PER, 3, 12, 33, kernel=kernel, tiling=tiling)
    assert np.array_equal(got, ref) and np.array_equal(gc, rc)


def test_domain_generic_scheme(rk):
    """Dormand-Prince 5 with second neighbours: 12 sites of reach per step (6 needed stages x
    2; the seventh stage feeds nothing), ghost 28 gives two steps per exchange; the ghost bonds
    of the second-neighbour energy end inside the ghosts."""
    A, b, _ = P.TABLEAUX["dopri5"]

    def setup(h):
        rk.rk4_chain_set_tableau(h, A, b)
        rk.rk4_chain_set_coupling2(h, 0.4)

    for model, bc in [(ROE, PER), (HAR, FIX)]:
        D = 3 if model == ROE else 2
        y0 = ci.uniform_state(7001, D, seed=730 + model)
        ref, _, re = whole(rk, y0, model, 0, bc, 15, setup)
        got, _, ge = domain(rk, y0, model, 0, bc, 4, 28, 15, setup=setup)
        assert np.array_equal(got, ref)
        assert ge == pytest.approx(re, rel=1e-13)


def test_domain_full_size(rk):
    """N = 2^22 over 4 parts, FP64, the default blocked tiling: bitwise against the whole chain."""
    y0 = ci.uniform_state(1 << 22, 3, seed=740)
    ref, _, re = whole(rk, y0, ROE, 0, PER, 24)
    got, _, ge = domain(rk, y0, ROE, 0, PER, 4, 32, 24)
    assert np.array_equal(got, ref)
    assert ge == pytest.approx(re, rel=1e-13)


def test_domain_errors(rk):
    import torch
    d = rk.rk4_domain_create(ROE, 0, 4000, 0.01, PER, 4, 8)
    try:
        rows, D = rk.rk4_domain_shape(d)
        st = torch.zeros((rows, D), dtype=torch.float64, device="cuda")
        wsb = rk.rk4_domain_workspace_bytes(d)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        with pytest.raises(rk.RK4Error) as ei:
            rk.rk4_domain_integrate(d, st, None, ws, 3, ws_bytes=wsb - 256)
        assert ei.value.code == rk.RK4_ENOMEM_WS
        with pytest.raises(rk.RK4Error) as ei:  # comp given for FP64
            rk.rk4_domain_integrate(d, st, st, ws, 3)
        assert ei.value.code == rk.RK4_EINVAL
        h = rk.rk4_domain_chain(d)
        A, b, _ = P.TABLEAUX["dopri5"]
        rk.rk4_chain_set_tableau(h, A, b)  # reach 6 <= ghost 8: one step per exchange
        rk.rk4_domain_integrate(d, st, None, ws, 2)
        rk.rk4_chain_set_coupling2(h, 0.3)  # reach 12 > 8
        with pytest.raises(rk.RK4Error) as ei:
            rk.rk4_domain_integrate(d, st, None, ws, 1)
        assert ei.value.code == rk.RK4_EUNSUPPORTED
        rk.rk4_chain_set_coupling2(h, 0.0)
        rk.rk4_chain_set_tableau(h, None)
        sp = torch.ones((rows, 4), dtype=torch.float64, device="cuda")
        rk.rk4_chain_set_site_params(h, sp)
        with pytest.raises(rk.RK4Error) as ei:
            rk.rk4_domain_integrate(d, st, None, ws, 1)
        assert ei.value.code == rk.RK4_EUNSUPPORTED
        rk.rk4_chain_set_site_params(h, None)
        part = rk.rk4_domain_part(d, 2)
        st[part["row"] + part["ghost_left"] + 5, 1] = float("nan")  # a site, not a ghost
        with pytest.raises(rk.RK4Error) as ei:
            rk.rk4_domain_energy(d, st, None, ws)
        assert ei.value.code == rk.RK4_ENONFINITE
    finally:
        rk.rk4_domain_destroy(d)


def test_domain_guard_bands(rk):
    """Canary margins around the domain state, compensation, whole-chain buffers and workspace
    stay intact through scatter, integrate, energy and gather."""
    import torch
    from test_gpu_guard import Guarded
    n, D = 9001, 3
    d = rk.rk4_domain_create(ROE, 1, n, 0.01, FIX, 3, 8, part_lengths=[8, 4000, 4993])
    try:
        rows, _ = rk.rk4_domain_shape(d)
        bufs = [Guarded(n * D * 4), Guarded(n * D * 4), Guarded(rows * D * 4), Guarded(rows * D * 4)]
        cst, ccp, st, cp = (g.typed(torch.float32, s) for g, s in zip(bufs, [(n, D), (n, D), (rows, D), (rows, D)]))
        cst.copy_(torch.from_numpy(ci.uniform_state(n, D, seed=750)).float())
        ccp.zero_()
        cp.zero_()
        wsb = rk.rk4_domain_workspace_bytes(d)
        gw = Guarded(wsb)
        bufs.append(gw)
        rk.rk4_domain_scatter(d, cst, ccp, st, cp)
        rk.rk4_domain_integrate(d, st, cp, gw.view, 17, ws_bytes=wsb)
        rk.rk4_domain_energy(d, st, cp, gw.view, ws_bytes=wsb)
        rk.rk4_domain_gather(d, st, cp, cst, ccp)
        torch.cuda.synchronize()
        assert all(b.intact() for b in bufs)
    finally:
        rk.rk4_domain_destroy(d)


def test_domain_graph_replay_and_recapture(rk):
    """Repeated calls replay the captured graph of 8 whole periods; between replays the
    leftover periods and a remainder of fewer steps run other launch plans (a batch's tables
    differ per plan), and a tiling change forces a new capture: state and compensation stay
    bit-identical to the undivided chain."""
    import torch
    n, ghost = 30011, 8  # RK4 reaches 4 sites per step: period 2
    y0 = ci.uniform_state(n, 3, seed=760).astype(np.float32)
    d = rk.rk4_domain_create(ROE, 1, n, 0.01, PER, 5, ghost, part_lengths=[6000, 12, 9000, 7999, 7000])
    try:
        h = rk.rk4_domain_chain(d)
        rk.rk4_chain_set_tiling(h, 256, 4, 2)
        rows, D = rk.rk4_domain_shape(d)
        cst, ccp = tensors(y0, 1)
        st = torch.zeros((rows, D), dtype=torch.float32, device="cuda")
        cp = torch.zeros_like(st)
        ws = torch.empty(rk.rk4_domain_workspace_bytes(d), dtype=torch.uint8, device="cuda")
        rk.rk4_domain_scatter(d, cst, ccp, st, cp)
        for _ in range(3):  # 21 steps: one 8-period graph chunk, 2 more periods, 1 remainder step
            t = rk.rk4_domain_integrate(d, st, cp, ws, 21)
        assert t == pytest.approx(63 * 0.01, rel=1e-15)
        rk.rk4_domain_gather(d, st, cp, cst, ccp)
        torch.cuda.synchronize()
        ref, rc, _ = whole(rk, y0, ROE, 1, PER, 63)
        assert np.array_equal(cst.cpu().numpy(), ref) and np.array_equal(ccp.cpu().numpy(), rc)
        rk.rk4_chain_set_tiling(h, 128, 8, 3)  # new configuration: captured again
        for _ in range(2):
            t = rk.rk4_domain_integrate(d, st, cp, ws, 21)
        assert t == pytest.approx(105 * 0.01, rel=1e-15)
        rk.rk4_domain_gather(d, st, cp, cst, ccp)
        torch.cuda.synchronize()
        ref, rc, _ = whole(rk, y0, ROE, 1, PER, 105)
        assert np.array_equal(cst.cpu().numpy(), ref) and np.array_equal(ccp.cpu().numpy(), rc)
    finally:
        rk.rk4_domain_destroy(d)
