"""GPU parity of the generic explicit-RK kernels (any tableau up to 7 stages, nearest or
next-nearest-neighbour coupling) against the oracle, and bit identity between the generic
one-stage-per-launch scheme and the generic temporally blocked kernel."""
import numpy as np
import pytest

import chain_inputs as ci
import closed_form as cf
import oracle
from tolerances import FP32_KAHAN_TOL
import oracle_pins as P

pytestmark = pytest.mark.gpu

PER, FIX = 0, 1
ROE, HAR = 0, 1
TABLEAUX = list(P.TABLEAUX.items())


@pytest.fixture(scope="module")
def rk():
    import torch
    import paper_1412_0544_gb300 as m
    assert torch.cuda.is_available()
    return m


def run(rk, y0, *, model=ROE, bc=PER, prec=0, nsteps=10, A=None, b=None, kappa=1.0, kappa2=0.0, kernel=None,
        tiling=None, lengths=None, kappas=None, bcs=None, dt=0.01, with_comp=False):
    import torch
    params = dict(kappa=kappa, omega0=0.8)
    if lengths is not None:
        h = rk.rk4_batch_create(model, prec, lengths, kappas, bcs, dt, params)
    else:
        h = rk.rk4_chain_create(model, prec, y0.shape[0], dt, bc, params)
    try:
        if A is not None:
            rk.rk4_chain_set_tableau(h, A, b)
        if kappa2:
            rk.rk4_chain_set_coupling2(h, kappa2)
        if kernel is not None:
            rk.rk4_chain_set_kernel(h, kernel)
        if tiling is not None:
            rk.rk4_chain_set_tiling(h, *tiling)
        dtype = torch.float32 if prec else torch.float64
        st = torch.from_numpy(np.ascontiguousarray(y0)).to(dtype).cuda()
        cp = torch.zeros_like(st) if prec else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
        torch.cuda.synchronize()
        out = st.double().cpu().numpy()
        if with_comp:
            return out, cp.double().cpu().numpy()
        return out
    finally:
        rk.rk4_chain_destroy(h)


@pytest.mark.parametrize("name,tab", TABLEAUX, ids=[t[0] for t in TABLEAUX])
@pytest.mark.parametrize("model,bc,kappa2", [(ROE, PER, 0.0), (ROE, FIX, 0.7), (HAR, FIX, 0.0), (HAR, PER, 0.6)])
def test_generic_vs_oracle_and_bitwise(rk, name, tab, model, bc, kappa2):
    A, b, _ = tab
    D = 3 if model == ROE else 2
    y0 = ci.uniform_state(3001, D, seed=300 + model + 2 * bc)
    nsteps = 60
    ref = oracle.rk_integrate(y0, A, b, model, bc, 0.01, nsteps,
                              oracle.params(kappa=1.0, omega0=0.8, kappa2=kappa2))
    st = run(rk, y0, model=model, bc=bc, nsteps=nsteps, A=A, b=b, kappa2=kappa2, kernel=rk.RK4_KERNEL_STAGED)
    assert cf.rel_inf(st, ref) <= 1e-12
    for tiling in [(128, 2, 1), (64, 4, 3), (256, 2, 2)]:
        got = run(rk, y0, model=model, bc=bc, nsteps=nsteps, A=A, b=b, kappa2=kappa2,
                  kernel=rk.RK4_KERNEL_BLOCKED, tiling=tiling)
        assert np.array_equal(got, st), tiling


def test_generic_rk4_close_to_specialised_rk4(rk):
    """The generic kernel with the classical tableau agrees with the RK4 kernels to rounding."""
    y0 = ci.uniform_state(20000, 3, seed=310)
    a = run(rk, y0, nsteps=200)
    b = run(rk, y0, nsteps=200, A=oracle.RK4_A, b=oracle.RK4_B)
    assert cf.rel_inf(b, a) <= 1e-13


def test_nnn_harmonic_closed_form(rk):
    y0 = ci.uniform_state(1024, 2, seed=320)
    got = run(rk, y0, model=HAR, bc=PER, nsteps=500, kappa=1.1, kappa2=0.6, tiling=(128, 4, 4))
    ref = cf.rk4_modal(y0, PER, 1.1, 0.8, 0.01, 500, kappa2=0.6)
    assert cf.rel_inf(got, ref) <= 1e-12


def test_nnn_dependency_cone(rk):
    """Second-neighbour coupling: one perturbed site changes exactly 8 sites per step each way."""
    n, site = 3000, 1500
    y0 = ci.uniform_state(n, 3, seed=330)
    y1 = y0.copy()
    y1[site, 0] += 0.5
    for m in (1, 2):
        a = run(rk, y0, bc=FIX, nsteps=m, dt=0.1, kappa=5.0, kappa2=10.0, tiling=(128, 4, 1))
        bb = run(rk, y1, bc=FIX, nsteps=m, dt=0.1, kappa=5.0, kappa2=10.0, tiling=(128, 4, 1))
        changed = np.nonzero(np.any(a != bb, axis=1))[0]
        assert changed.min() == site - 8 * m and changed.max() == site + 8 * m


@pytest.mark.parametrize("bc", [PER, FIX])
def test_nnn_energy_reduction(rk, bc):
    import torch
    y0 = ci.uniform_state(70001, 2, seed=340 + bc)
    h = rk.rk4_chain_create(HAR, rk.RK4_FP64, y0.shape[0], 0.01, bc, dict(kappa=1.1, omega0=0.9))
    rk.rk4_chain_set_coupling2(h, 0.45)
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    e = rk.rk4_chain_energy(h, torch.from_numpy(y0).cuda(), None, ws)[0]
    ref = oracle.energy_harmonic(y0, bc, oracle.params(kappa=1.1, omega0=0.9, kappa2=0.45))
    rk.rk4_chain_destroy(h)
    assert abs(e - ref) <= 1e-12 * abs(ref)


def test_generic_fp32_kahan(rk):
    A, b, _ = P.TABLEAUX["dopri5"]
    y0 = ci.uniform_state(8192, 3, seed=350).astype(np.float32)
    st, cst = run(rk, y0, prec=1, nsteps=300, A=A, b=b, kappa2=0.5, kernel=rk.RK4_KERNEL_STAGED, with_comp=True)
    got, cgot = run(rk, y0, prec=1, nsteps=300, A=A, b=b, kappa2=0.5, tiling=(128, 4, 4), with_comp=True)
    assert np.array_equal(got, st) and np.array_equal(cgot, cst)
    ref = oracle.rk_integrate(y0.astype(np.float64), A, b, ROE, PER, 0.01, 300, oracle.params(kappa2=0.5))
    err = cf.rel_inf(st - cst, ref)
    print(f"FP32-Kahan dopri5 + NNN, 300 steps: rel err vs FP64 oracle {err:.2e}")
    assert err <= FP32_KAHAN_TOL


@pytest.mark.parametrize("shape", ["dopri5", "rk4"])
@pytest.mark.parametrize("model,bc,kappa2", [(ROE, FIX, 0.7), (ROE, PER, 0.0), (HAR, FIX, 0.0), (HAR, PER, 0.6)])
def test_generic_fp32_compiled_shapes_bitwise(rk, shape, model, bc, kappa2):
    """The tableau shapes with compiled FP32 tile kernels (4 sites per thread) issue their
    arithmetic on packed pairs of sites; every model, boundary (fixed ends mask ghost sites) and
    coupling range must still give the scalar one-stage-per-launch kernel's bits, state and
    compensation alike."""
    A, b, _ = P.TABLEAUX[shape]
    D = 3 if model == ROE else 2
    y0 = ci.uniform_state(5003, D, seed=370 + model + 2 * bc).astype(np.float32)
    nsteps = 41
    st, cst = run(rk, y0, model=model, bc=bc, prec=1, nsteps=nsteps, A=A, b=b, kappa2=kappa2,
                  kernel=rk.RK4_KERNEL_STAGED, with_comp=True)
    for tiling in [(128, 4, 2), (64, 4, 3), (512, 4, 1)]:
        got, cgot = run(rk, y0, model=model, bc=bc, prec=1, nsteps=nsteps, A=A, b=b, kappa2=kappa2,
                        kernel=rk.RK4_KERNEL_BLOCKED, tiling=tiling, with_comp=True)
        assert np.array_equal(got, st) and np.array_equal(cgot, cst), tiling
    ref = oracle.rk_integrate(y0.astype(np.float64), A, b, model, bc, 0.01, nsteps,
                              oracle.params(kappa=1.0, omega0=0.8, kappa2=kappa2))
    assert cf.rel_inf(st - cst, ref) <= FP32_KAHAN_TOL


def test_generic_fp32_batch_bitwise(rk):
    """Uneven FP32 chains with the Dormand-Prince 5 shape and second neighbours (packed pairs,
    per-chain coupling, mixed ends) against the staged kernel, bit for bit."""
    A, b, _ = P.TABLEAUX["dopri5"]
    lengths, kappa, bcs = ci.batch_spec(30, seed=380, nmin=1, nmax=3000)
    y0 = ci.uniform_state(int(lengths.sum()), 3, seed=381).astype(np.float32)
    st, cst = run(rk, y0, prec=1, nsteps=33, A=A, b=b, kappa2=0.4, lengths=lengths, kappas=kappa, bcs=bcs,
                  kernel=rk.RK4_KERNEL_STAGED, with_comp=True)
    for tiling in [(128, 4, 2), (256, 4, 4)]:
        got, cgot = run(rk, y0, prec=1, nsteps=33, A=A, b=b, kappa2=0.4, lengths=lengths, kappas=kappa, bcs=bcs,
                        kernel=rk.RK4_KERNEL_BLOCKED, tiling=tiling, with_comp=True)
        assert np.array_equal(got, st) and np.array_equal(cgot, cst), tiling


def test_generic_batch(rk):
    A, b, _ = P.TABLEAUX["kutta3"]
    lengths, kappa, bcs = ci.batch_spec(40, seed=360, nmin=1, nmax=2000)
    y0 = ci.uniform_state(int(lengths.sum()), 3, seed=361)
    st = run(rk, y0, nsteps=40, A=A, b=b, kappa2=0.3, lengths=lengths, kappas=kappa, bcs=bcs,
             kernel=rk.RK4_KERNEL_STAGED)
    got = run(rk, y0, nsteps=40, A=A, b=b, kappa2=0.3, lengths=lengths, kappas=kappa, bcs=bcs,
              tiling=(128, 2, 2))
    assert np.array_equal(got, st)
    off = 0
    for n, k, bc in zip(lengths, kappa, bcs):
        ref = oracle.rk_integrate(y0[off:off + n], A, b, ROE, int(bc), 0.01, 40,
                                  oracle.params(kappa=float(k), kappa2=0.3))
        assert cf.rel_inf(st[off:off + n], ref) <= 1e-12
        off += n


def test_generic_persistent_unsupported(rk):
    import torch
    h = rk.rk4_chain_create(ROE, rk.RK4_FP64, 1000, 0.01, PER)
    rk.rk4_chain_set_coupling2(h, 0.5)
    rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_PERSISTENT)
    st = torch.zeros((1000, 3), dtype=torch.float64, device="cuda")
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    with pytest.raises(rk.RK4Error) as ei:
        rk.rk4_chain_integrate(h, st, None, ws, 2)
    assert ei.value.code == rk.RK4_EUNSUPPORTED
    rk.rk4_chain_destroy(h)
