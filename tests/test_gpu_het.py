"""GPU parity of heterogeneous chains (Eq. (1) of the paper: site-dependent f_i and g_i through
per-site parameters) against the oracle, bit identity between the staged and blocked kernels,
and bit identity with the homogeneous kernels when every site has the same parameters."""
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


@pytest.fixture(scope="module")
def rk():
    import torch
    import paper_1412_0544_gb300 as m
    assert torch.cuda.is_available()
    return m


def run(rk, y0, sp, *, model=ROE, bc=PER, prec=0, nsteps=10, kernel=None, tiling=None, lengths=None,
        kappas=None, bcs=None, with_comp=False):
    import torch
    dtype = torch.float32 if prec else torch.float64
    if lengths is not None:
        h = rk.rk4_batch_create(model, prec, lengths, kappas, bcs, 0.01)
    else:
        h = rk.rk4_chain_create(model, prec, y0.shape[0], 0.01, bc)
    try:
        spd = None
        if sp is not None:
            spd = torch.from_numpy(np.ascontiguousarray(sp)).to(dtype).cuda()
            rk.rk4_chain_set_site_params(h, spd)
        if kernel is not None:
            rk.rk4_chain_set_kernel(h, kernel)
        if tiling is not None:
            rk.rk4_chain_set_tiling(h, *tiling)
        st = torch.from_numpy(np.ascontiguousarray(y0)).to(dtype).cuda()
        cp = torch.zeros_like(st) if prec else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
        torch.cuda.synchronize()
        out = st.double().cpu().numpy()
        return (out, cp.double().cpu().numpy()) if with_comp else out
    finally:
        rk.rk4_chain_destroy(h)


@pytest.mark.parametrize("model,bc", [(ROE, PER), (ROE, FIX), (HAR, PER), (HAR, FIX)])
def test_het_vs_oracle_and_bitwise(rk, model, bc):
    D = 3 if model == ROE else 2
    n = 5003
    y0 = ci.uniform_state(n, D, seed=400 + model + 2 * bc)
    sp = P.het_params(n, model, 401 + bc)
    ref = oracle.rk4_integrate_het(y0, sp, model, bc, 0.01, 80)
    st = run(rk, y0, sp, model=model, bc=bc, nsteps=80, kernel=rk.RK4_KERNEL_STAGED)
    assert cf.rel_inf(st, ref) <= 1e-12
    for tiling in [(256, 2, 1), (128, 4, 4), (256, 2, 8), (512, 4, 2)]:
        got = run(rk, y0, sp, model=model, bc=bc, nsteps=80, tiling=tiling)
        assert np.array_equal(got, st), tiling


def test_uniform_parameters_equal_homogeneous_bitwise(rk):
    """With the same parameters at every site the heterogeneous kernels perform exactly the
    homogeneous kernels' operations."""
    n = 10007
    y0 = ci.uniform_state(n, 3, seed=410)
    sp = np.tile([0.2, 1.0, 9.0, 1.0], (n, 1))
    a = run(rk, y0, sp, nsteps=37, tiling=(256, 2, 2))
    b = run(rk, y0, None, nsteps=37, tiling=(256, 4, 4))
    assert np.array_equal(a, b)


def test_het_harmonic_eigen_closed_form(rk):
    """Site-dependent frequencies with uniform coupling: the GPU against the eigen-decomposition
    closed form directly."""
    n, nsteps, kappa = 64, 800, 1.3
    y0 = ci.uniform_state(n, 2, seed=420)
    sp = P.het_params(n, HAR, 421)
    sp[:, 1] = kappa
    L = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    L[0, -1] += 1.0
    L[-1, 0] += 1.0
    lam, V = np.linalg.eigh(np.diag(sp[:, 0]) - kappa * L)
    w = np.sqrt(lam)
    h = w * 0.01
    alpha, beta = 1 - h ** 2 / 2 + h ** 4 / 24, 1 - h ** 2 / 6
    rho, theta = alpha ** 2 + (beta * h) ** 2, np.arctan2(beta * h, alpha)
    qh, sh = V.T @ y0[:, 0], (V.T @ y0[:, 1]) / w
    amp, ang = rho ** (nsteps / 2), nsteps * theta
    ref = np.stack([V @ (amp * (np.cos(ang) * qh + np.sin(ang) * sh)),
                    V @ (amp * (-np.sin(ang) * qh + np.cos(ang) * sh) * w)], axis=1)
    got = run(rk, y0, sp, model=HAR, bc=PER, nsteps=nsteps, tiling=(64, 2, 4))
    assert cf.rel_inf(got, ref) <= 1e-12


def test_het_fp32_kahan(rk):
    n = 40000
    y0 = ci.uniform_state(n, 3, seed=430).astype(np.float32)
    sp = P.het_params(n, ROE, 431).astype(np.float32)
    st, cst = run(rk, y0, sp, prec=1, nsteps=500, kernel=rk.RK4_KERNEL_STAGED, with_comp=True)
    for tiling in [(256, 4, 8), (256, 2, 8)]:  # per-thread and warp neighbour exchange
        got, cgot = run(rk, y0, sp, prec=1, nsteps=500, tiling=tiling, with_comp=True)
        assert np.array_equal(got, st) and np.array_equal(cgot, cst), tiling
    ref = oracle.rk4_integrate_het(y0.astype(np.float64), sp.astype(np.float64), ROE, PER, 0.01, 500)
    err = cf.rel_inf(st - cst, ref)
    print(f"heterogeneous FP32-Kahan, 500 steps: rel err vs FP64 oracle {err:.2e}")
    assert err <= FP32_KAHAN_TOL


@pytest.mark.parametrize("model,bc", [(ROE, FIX), (HAR, PER), (HAR, FIX)])
def test_het_fp32_kahan_models_and_ends_bitwise(rk, model, bc):
    """FP32-Kahan heterogeneous tiles on packed pairs of sites, whose per-site coefficients
    are read per stage from shared memory in pair order: both models (four and two per-site
    coefficients), fixed ends (ghost sites), against the staged kernel bit for bit."""
    D = 3 if model == ROE else 2
    n = 20011
    y0 = ci.uniform_state(n, D, seed=435 + model + 2 * bc).astype(np.float32)
    sp = P.het_params(n, model, 436 + bc).astype(np.float32)
    st, cst = run(rk, y0, sp, model=model, bc=bc, prec=1, nsteps=64, kernel=rk.RK4_KERNEL_STAGED, with_comp=True)
    for tiling in [(256, 4, 4), (128, 2, 8), (64, 4, 2)]:
        got, cgot = run(rk, y0, sp, model=model, bc=bc, prec=1, nsteps=64, tiling=tiling, with_comp=True)
        assert np.array_equal(got, st) and np.array_equal(cgot, cst), tiling
    ref = oracle.rk4_integrate_het(y0.astype(np.float64), sp.astype(np.float64), model, bc, 0.01, 64)
    assert cf.rel_inf(st - cst, ref) <= FP32_KAHAN_TOL


def test_het_batch(rk):
    lengths, kappa, bcs = ci.batch_spec(50, seed=440, nmin=1, nmax=3000)
    total = int(lengths.sum())
    y0 = ci.uniform_state(total, 3, seed=441)
    sp = P.het_params(total, ROE, 442)
    st = run(rk, y0, sp, nsteps=50, lengths=lengths, kappas=kappa, bcs=bcs, kernel=rk.RK4_KERNEL_STAGED)
    got = run(rk, y0, sp, nsteps=50, lengths=lengths, kappas=kappa, bcs=bcs, kernel=rk.RK4_KERNEL_BLOCKED,
              tiling=(256, 2, 4))
    assert np.array_equal(got, st)
    off = 0
    for n, bc in zip(lengths, bcs):
        ref = oracle.rk4_integrate_het(y0[off:off + n], sp[off:off + n], ROE, int(bc), 0.01, 50)
        assert cf.rel_inf(st[off:off + n], ref) <= 1e-12
        off += n


def test_het_unsupported_paths(rk):
    import torch
    n = 1000
    h = rk.rk4_chain_create(HAR, rk.RK4_FP64, n, 0.01, PER)
    sp = torch.ones((n, 2), dtype=torch.float64, device="cuda")
    rk.rk4_chain_set_site_params(h, sp)
    st = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    with pytest.raises(rk.RK4Error) as ei:
        rk.rk4_chain_energy(h, st, None, ws)
    assert ei.value.code == rk.RK4_EUNSUPPORTED
    rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_PERSISTENT)
    with pytest.raises(rk.RK4Error) as ei:
        rk.rk4_chain_integrate(h, st, None, ws, 1)
    assert ei.value.code == rk.RK4_EUNSUPPORTED
    rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_AUTO)
    rk.rk4_chain_set_coupling2(h, 0.5)
    with pytest.raises(rk.RK4Error) as ei:
        rk.rk4_chain_integrate(h, st, None, ws, 1)
    assert ei.value.code == rk.RK4_EUNSUPPORTED
    rk.rk4_chain_destroy(h)
