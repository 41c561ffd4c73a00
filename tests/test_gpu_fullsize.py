"""GPU parity at the workload sizes (N = 2^24 and 2^27, 1000 / 200 steps, 4096-chain batch).

The oracle cannot integrate 2^27 sites for 1000 steps in seconds, but it can compute any one
site exactly: after T steps site i depends only on sites i - 4T .. i + 4T (four stages per
step, each reaching one neighbour further -- the paper's overlap argument, Sec. 2.3).  So the
oracle integrates the 8T + 1-site window around each sampled site with fixed (artificial)
ends and the window's centre is the full chain's value bit for bit.  Inputs on both sides come
from the same counter generator (device fill vs host generator, checked bit-exact elsewhere).
"""
import numpy as np
import pytest

import chain_inputs as ci
import closed_form as cf
import oracle
from tolerances import FP32_KAHAN_TOL

pytestmark = pytest.mark.gpu

SEED = ci.DEFAULT_SEED


@pytest.fixture(scope="module")
def rk():
    import torch
    import paper_1412_0544_gb300 as m
    assert torch.cuda.is_available()
    return m


def host_sites(idx, D):
    """Initial values of the given global site indices (stream 0 of the generator)."""
    idx = np.asarray(idx, dtype=np.int64)
    out = np.empty((idx.size, D))
    # contiguous runs keep this cheap
    for d in range(D):
        j = idx * D + d
        out[:, d] = 2.0 * _u01_at(j) - 1.0
    return out


def _u01_at(j):
    z = ci.splitmix64(np.asarray(j, dtype=np.uint64) ^ np.uint64(SEED))
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def cone_oracle(i, n, T, bc, D=3, model=oracle.ROESSLER, prm=None, dtype=np.float64):
    """Oracle value of site i of an n-site chain after T steps, from its dependency cone."""
    r = 4 * T
    if bc == oracle.PERIODIC:
        idx = np.arange(i - r, i + r + 1) % n
        centre = r
        y0 = host_sites(idx, D)
    else:
        lo, hi = max(0, i - r), min(n, i + r + 1)
        idx = np.arange(lo, hi)
        centre = i - lo
        y0 = host_sites(idx, D)
        # a window end that is a true chain end keeps its fixed boundary; an artificial end
        # only spoils sites further than 4T from the centre
    if dtype == np.float32:
        y0 = y0.astype(np.float32).astype(np.float64)
    out = oracle.rk4_integrate(y0, model, oracle.FIXED, 0.01, T, prm)
    return out[centre]


def sample_sites(n, G):
    s = {0, 1, 2, n - 1, n - 2, n // 2, G - 1, G, G + 1, 3 * G - 1, n - G, (n // G) * G}
    rng = np.random.default_rng(5)
    s.update(int(x) for x in rng.integers(0, n, 4))
    return sorted(x for x in s if 0 <= x < n)


def run_chain(rk, n, bc, prec, T, tiling=None, autotune=False, kernel=None):
    import torch
    h = rk.rk4_chain_create(rk.RK4_ROESSLER, prec, n, 0.01, bc)
    if kernel is not None:
        rk.rk4_chain_set_kernel(h, kernel)
    dt = torch.float64 if prec == rk.RK4_FP64 else torch.float32
    st = torch.empty((n, 3), dtype=dt, device="cuda")
    rk.rk4_fill_uniform(st, n * 3, SEED, 0, prec)
    cp = torch.zeros_like(st) if prec == rk.RK4_FP32_KAHAN else None
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    if autotune:
        rk.rk4_chain_autotune(h, st.clone(), cp.clone() if cp is not None else None, ws, 16)
    elif tiling:
        rk.rk4_chain_set_tiling(h, *tiling)
    til = rk.rk4_chain_get_tiling(h)
    rk.rk4_chain_integrate(h, st, cp, ws, T)
    torch.cuda.synchronize()
    assert rk.rk4_chain_status(h, ws) == rk.RK4_OK
    rk.rk4_chain_destroy(h)
    return st, cp, til


def test_bench_workload_fp64_2e24_1000_steps(rk):
    """The benchmark's launch configuration (autotuned tiling), sampled against the oracle."""
    n, T = 1 << 24, 1000
    st, _, til = run_chain(rk, n, rk.RK4_PERIODIC, rk.RK4_FP64, T, autotune=True)
    sites = sample_sites(n, til["G"])[:10]
    got = st[sites].cpu().numpy()
    ref = np.array([cone_oracle(i, n, T, oracle.PERIODIC) for i in sites])
    err = cf.rel_inf(got, ref)
    print(f"N=2^24 FP64 1000 steps tiling {til}: sampled rel err {err:.2e}")
    assert err <= 1e-12


def test_fixed_fp64_2e27_200_steps(rk):
    """The benchmark's workload and launch configuration (fixed ends, N = 2^27, 200 steps,
    autotuned tiling), sampled against the oracle."""
    n, T = 1 << 27, 200
    st, _, til = run_chain(rk, n, rk.RK4_FIXED, rk.RK4_FP64, T, autotune=True)
    sites = sample_sites(n, til["G"])
    got = st[sites].cpu().numpy()
    ref = np.array([cone_oracle(i, n, T, oracle.FIXED) for i in sites])
    assert cf.rel_inf(got, ref) <= 1e-12


def test_fp32_kahan_2e27_1000_steps(rk):
    """FP32-Kahan at N = 2^27: each sampled site equals, bit for bit, the same kernel run on
    that site's 8T+1-site dependency window (a property that holds at any size), and lies
    within the stated error of the FP64 oracle started from the same FP32 values."""
    import torch
    n, T = 1 << 27, 1000
    st, cp, til = run_chain(rk, n, rk.RK4_PERIODIC, rk.RK4_FP32_KAHAN, T, tiling=(128, 8, 16))
    sites = sample_sites(n, til["G"])[:6]
    for i in sites[:3]:
        r = 4 * T
        win = host_sites(np.arange(i - r, i + r + 1) % n, 3).astype(np.float32)
        h = rk.rk4_chain_create(rk.RK4_ROESSLER, rk.RK4_FP32_KAHAN, win.shape[0], 0.01, rk.RK4_FIXED)
        ws_ = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        w = torch.from_numpy(win).cuda()
        wc = torch.zeros_like(w)
        rk.rk4_chain_integrate(h, w, wc, ws_, T)
        torch.cuda.synchronize()
        rk.rk4_chain_destroy(h)
        assert torch.equal(w[r], st[i]) and torch.equal(wc[r], cp[i]), i
    got = (st[sites].double() - cp[sites].double()).cpu().numpy()
    ref = np.array([cone_oracle(i, n, T, oracle.PERIODIC, dtype=np.float32) for i in sites])
    err = cf.rel_inf(got, ref)
    print(f"N=2^27 FP32-Kahan 1000 steps: sampled rel err vs FP64 oracle {err:.2e}")
    assert err <= FP32_KAHAN_TOL


def test_batch_4096_chains_1000_steps(rk):
    import torch
    lengths, kappa, bcs = ci.batch_spec(4096, seed=SEED)
    total = int(lengths.sum())
    offs = np.concatenate(([0], np.cumsum(lengths)))
    picks = [int(np.argmin(lengths)), int(np.argmax(lengths)), 0, 1, 2047, 4095]
    for prec in (rk.RK4_FP64, rk.RK4_FP32_KAHAN):
        h = rk.rk4_batch_create(rk.RK4_ROESSLER, prec, lengths, kappa, bcs, 0.01)
        dt = torch.float64 if prec == rk.RK4_FP64 else torch.float32
        st = torch.empty((total, 3), dtype=dt, device="cuda")
        rk.rk4_fill_uniform(st, total * 3, SEED, 0, prec)
        cp = torch.zeros_like(st) if prec == rk.RK4_FP32_KAHAN else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_set_tiling(h, 256, 4, 4)
        rk.rk4_chain_integrate(h, st, cp, ws, 1000)
        torch.cuda.synchronize()
        assert rk.rk4_chain_status(h, ws) == rk.RK4_OK
        for c in picks:
            a, b = offs[c], offs[c + 1]
            y0 = host_sites(np.arange(a, b), 3)
            if prec == rk.RK4_FP32_KAHAN:
                y0 = y0.astype(np.float32).astype(np.float64)
            ref = oracle.rk4_integrate(y0, oracle.ROESSLER, int(bcs[c]), 0.01, 1000,
                                       oracle.params(kappa=float(kappa[c])))
            got = st[a:b].double()
            if cp is not None:
                got = got - cp[a:b].double()
            err = cf.rel_inf(got.cpu().numpy(), ref)
            assert err <= (1e-12 if prec == rk.RK4_FP64 else FP32_KAHAN_TOL), (c, int(lengths[c]), err)
        rk.rk4_chain_destroy(h)


# Tilings of the full-size bitwise check: for each tile width W = block x v, one shape with the
# per-thread shared-memory exchange (4 or 8 sites per thread) and one with the warp-shuffle
# exchange (1 or 2 sites per thread), where the kernels are compiled for it.
FULLSIZE_SHAPES = {256: [(64, 4), (256, 1)], 512: [(128, 4), (256, 2)], 1024: [(256, 4), (512, 2)],
                   2048: [(512, 4), (256, 8)]}


def test_blocked_bitwise_equals_staged_2e24_1000_steps(rk):
    """Sec. 2.3: granularity with overlap gives the cluster's exact result.  At N = 2^24 and
    1000 steps, every tiling of the sweep (W = 256 .. 2048 sites per tile, k = 1, 2, 4, 8 steps
    per launch), the autotuned pick and the persistent kernel all produce the one-stage-per-launch
    kernel's state bit for bit."""
    import torch
    n, T = 1 << 24, 1000
    ref, _, _ = run_chain(rk, n, rk.RK4_PERIODIC, rk.RK4_FP64, T, kernel=rk.RK4_KERNEL_STAGED)
    checked = []
    for W, shapes in FULLSIZE_SHAPES.items():
        for block, v in shapes:
            for k in (1, 2, 4, 8):
                st, _, _ = run_chain(rk, n, rk.RK4_PERIODIC, rk.RK4_FP64, T, tiling=(block, v, k),
                                     kernel=rk.RK4_KERNEL_BLOCKED)
                assert torch.equal(st, ref), (block, v, k)
                checked.append((block, v, k))
                del st
    st, _, til = run_chain(rk, n, rk.RK4_PERIODIC, rk.RK4_FP64, T, autotune=True)
    assert torch.equal(st, ref), til
    del st
    st, _, til = run_chain(rk, n, rk.RK4_PERIODIC, rk.RK4_FP64, T, tiling=(256, 4, 4),
                           kernel=rk.RK4_KERNEL_PERSISTENT)
    assert torch.equal(st, ref), ("persistent", til)
    assert len(checked) == 32


def test_fp32_kahan_bitwise_equals_staged_2e24_1000_steps(rk):
    """The same for the FP32-Kahan path (state and compensation), on the tilings the autotuner
    picks from (k up to 16) and the persistent kernel."""
    import torch
    n, T = 1 << 24, 1000
    ref, cref, _ = run_chain(rk, n, rk.RK4_PERIODIC, rk.RK4_FP32_KAHAN, T, kernel=rk.RK4_KERNEL_STAGED)
    for tiling in [(256, 4, 1), (256, 4, 4), (512, 4, 16), (128, 8, 16), (256, 2, 8), (1024, 1, 2)]:
        st, cp, _ = run_chain(rk, n, rk.RK4_PERIODIC, rk.RK4_FP32_KAHAN, T, tiling=tiling,
                              kernel=rk.RK4_KERNEL_BLOCKED)
        assert torch.equal(st, ref) and torch.equal(cp, cref), tiling
    st, cp, til = run_chain(rk, n, rk.RK4_PERIODIC, rk.RK4_FP32_KAHAN, T, tiling=(256, 4, 8),
                            kernel=rk.RK4_KERNEL_PERSISTENT)
    assert torch.equal(st, ref) and torch.equal(cp, cref), ("persistent", til)
