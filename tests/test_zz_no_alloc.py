"""rk4_chain_energy_static: the energy / norm reduction for callers that cannot allocate
device memory (so cannot hand the library a workspace).  Its scratch is compiled into the
library; the result must agree with rk4_chain_energy, which uses the caller's workspace, on
two calls in a row (the shared scratch keeps the previous call's contents, so the second call
checks that nothing stale leaks in).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import chain_inputs as ci

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the relative tolerance the other FP64 reduction tests use


@pytest.fixture(scope="module")
def rk():
    import torch
    import paper_1412_0544_gb300 as m
    assert torch.cuda.is_available()
    return m


def _dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _agree(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.all(np.abs(a - b) <= TOL * np.maximum(np.abs(b), 1e-300))


def _static_no_alloc(rk, h, st, cp, check):
    """One rk4_chain_energy_static call; with `check`, the device's free memory is read right
    before and right after it (the device idle both times) and must not change.  Only calls
    after the first are checked: the first call on a device looks up the scratch array's
    address, and with lazy module loading that lookup is what brings the array (compiled into
    the library, not allocated by the call) onto the device."""
    import torch
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    got = rk.rk4_chain_energy_static(h, st, cp)
    torch.cuda.synchronize()
    if check:
        assert torch.cuda.mem_get_info()[0] == free_before
    return got


# (model, precision, D, boundary, second-neighbour coupling): the FP64 and FP32-Kahan
# reductions of both models, and the harmonic energy with second-neighbour bonds
SINGLE_CASES = [(0, 0, 3, 0, 0.0), (1, 0, 2, 1, 0.0), (0, 1, 3, 1, 0.0), (1, 1, 2, 0, 0.0), (1, 0, 2, 0, 0.45),
                (1, 1, 2, 1, 0.45)]


@pytest.mark.parametrize("model,prec,D,bc,kappa2", SINGLE_CASES)
def test_static_energy_matches_workspace_energy_single_chain(rk, model, prec, D, bc, kappa2):
    import torch
    n = 100003
    dtype = torch.float32 if prec == rk.RK4_FP32_KAHAN else torch.float64
    h = rk.rk4_chain_create(model, prec, n, 0.01, bc, dict(kappa=1.1, omega0=0.9))
    try:
        if kappa2:
            rk.rk4_chain_set_coupling2(h, kappa2)
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        for call, seed in enumerate((5, 6)):  # two calls in a row, different states
            st = _dev(ci.uniform_state(n, D, seed=seed + 10 * prec), dtype)
            cp = (st * 1e-8).contiguous() if prec == rk.RK4_FP32_KAHAN else None
            ref = rk.rk4_chain_energy(h, st, cp, ws)
            got = _static_no_alloc(rk, h, st, cp, check=call == 1)
            assert _agree(got, ref), (got, ref)
    finally:
        rk.rk4_chain_destroy(h)


def test_static_energy_matches_workspace_energy_batch_fp32(rk):
    import torch
    lengths, kappa, bcs = ci.batch_spec(300, seed=7, nmin=1, nmax=5000)
    total = int(lengths.sum())
    h = rk.rk4_batch_create(rk.RK4_HARMONIC, rk.RK4_FP32_KAHAN, lengths, kappa, bcs, 0.01)
    try:
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        st = _dev(ci.uniform_state(total, 2, seed=8), torch.float32)
        cp = (st * 1e-8).contiguous()
        for _ in range(2):
            ref = rk.rk4_chain_energy(h, st, cp, ws)
            got = rk.rk4_chain_energy_static(h, st, cp)
            assert got.shape == (300,)
            assert _agree(got, ref)
            rk.rk4_chain_integrate(h, st, cp, ws, 3)  # change the state between the calls
    finally:
        rk.rk4_chain_destroy(h)


def test_static_energy_largest_batch_and_rejection_beyond(rk):
    """8192 chains, the scratch array's limit, are reduced (twice, matching the workspace
    reduction); 8193 are rejected with RK4_EINVAL before anything is enqueued."""
    import torch
    lengths, kappa, bcs = ci.batch_spec(8192, seed=9, nmin=1, nmax=300)
    total = int(lengths.sum())
    h = rk.rk4_batch_create(rk.RK4_HARMONIC, rk.RK4_FP64, lengths, kappa, bcs, 0.01)
    try:
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        for call, seed in enumerate((10, 11)):
            st = _dev(ci.uniform_state(total, 2, seed=seed), torch.float64)
            ref = rk.rk4_chain_energy(h, st, None, ws)
            got = _static_no_alloc(rk, h, st, None, check=call == 1)
            assert got.shape == (8192,) and _agree(got, ref)
    finally:
        rk.rk4_chain_destroy(h)
    h = rk.rk4_batch_create(rk.RK4_ROESSLER, rk.RK4_FP64, np.full(8193, 2), np.ones(8193), np.zeros(8193), 0.01)
    try:
        st = torch.zeros((8193 * 2, 3), dtype=torch.float64, device="cuda")
        with pytest.raises(rk.RK4Error) as ei:
            rk.rk4_chain_energy_static(h, st, None)
        assert ei.value.code == rk.RK4_EINVAL
    finally:
        rk.rk4_chain_destroy(h)
