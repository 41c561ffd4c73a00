"""GPU parity: the CUDA kernels against the CPU oracle and against each other (needs a GB300).

* FP64 results match the oracle within 1e-12 (max-abs error relative to max |oracle|) after
  1000 steps -- the tolerance required of the FP64 path.
* The blocked kernel (every tiling), the fused k = 1 kernel and the persistent kernel are bit
  for bit equal to the one-stage-per-launch kernel.
* FP32-Kahan results are compared with the FP64 oracle started from the same FP32 values and
  their error is asserted below a stated bound.
Everything calls the library through its C ABI (ctypes binding); inputs come from the shared
seeded generator, expected values from the oracle only.
"""
import numpy as np
import pytest

import chain_inputs as ci
import closed_form as cf
import oracle
from tolerances import FP32_KAHAN_TOL

pytestmark = pytest.mark.gpu

PER, FIX = 0, 1
ROE, HAR = 0, 1


@pytest.fixture(scope="module")
def rk():
    import paper_1412_0544_gb300 as m  # fails loudly when the CUDA library is missing
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return m


@pytest.fixture(scope="module")
def gh(rk):
    import gpu_helpers
    return gpu_helpers


def rel(a, b):
    return cf.rel_inf(a, b)


# ---- FP64 against the oracle ----------------------------------------------------------

@pytest.mark.parametrize("bc", [PER, FIX])
def test_fp64_blocked_vs_oracle_65536_1000_steps(rk, gh, bc):
    """Plain FP64 RK4 on the paper's Roessler chain, N = 65536, dt = 0.01, 1000 steps."""
    y0 = ci.uniform_state(65536, 3)
    ref = oracle.rk4_integrate(y0, ROE, bc, 0.01, 1000)
    got = gh.gpu_run(y0, bc=bc, nsteps=1000)
    err = rel(got, ref)
    print(f"FP64 blocked vs oracle, bc={bc}: rel err {err:.3e}")
    assert err <= 1e-12


@pytest.mark.parametrize("model,bc", [(ROE, PER), (ROE, FIX), (HAR, PER), (HAR, FIX)])
def test_fp64_staged_vs_oracle(rk, gh, model, bc):
    D = 3 if model == ROE else 2
    y0 = ci.uniform_state(3001, D, seed=21 + bc)
    prm = oracle.params(kappa=1.3, omega0=0.8)
    params = dict(kappa=1.3, omega0=0.8)
    ref = oracle.rk4_integrate(y0, model, bc, 0.01, 200, prm)
    got = gh.gpu_run(y0, model=model, bc=bc, nsteps=200, params=params, kernel=rk.RK4_KERNEL_STAGED)
    assert rel(got, ref) <= 1e-12


def test_harmonic_gpu_vs_closed_form(rk, gh):
    """The GPU result against the normal-mode closed form directly (no oracle in between)."""
    for bc in (PER, FIX):
        y0 = ci.uniform_state(512, 2, seed=31 + bc)
        got = gh.gpu_run(y0, model=HAR, bc=bc, nsteps=1000, params=dict(kappa=1.3, omega0=0.7))
        ref = cf.rk4_modal(y0, bc, 1.3, 0.7, 0.01, 1000)
        assert rel(got, ref) <= 1e-12


# ---- bit identity between kernels ---------------------------------------------------

TILINGS = [(64, 1, 1), (128, 2, 1), (256, 4, 1), (256, 4, 2), (128, 8, 4), (512, 4, 8), (256, 8, 16),
           (1024, 1, 8), (512, 2, 16), (64, 4, 8)]


@pytest.fixture(scope="module")
def staged_refs(rk, gh):
    refs = {}
    for model in (ROE, HAR):
        D = 3 if model == ROE else 2
        for bc in (PER, FIX):
            y0 = ci.uniform_state(10007, D, seed=41 + 2 * model + bc)
            refs[(model, bc)] = (y0, gh.gpu_run(y0, model=model, bc=bc, nsteps=37, kernel=rk.RK4_KERNEL_STAGED))
    return refs


@pytest.mark.parametrize("tiling", TILINGS, ids=[f"b{b}v{v}k{k}" for b, v, k in TILINGS])
@pytest.mark.parametrize("model,bc", [(ROE, PER), (ROE, FIX), (HAR, PER), (HAR, FIX)])
def test_blocked_bitwise_equals_staged(rk, gh, staged_refs, tiling, model, bc):
    y0, ref = staged_refs[(model, bc)]
    got = gh.gpu_run(y0, model=model, bc=bc, nsteps=37, kernel=rk.RK4_KERNEL_BLOCKED, tiling=tiling)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("tiling", [(256, 4, 1), (128, 8, 4), (512, 2, 8)])
@pytest.mark.parametrize("model,bc", [(ROE, PER), (ROE, FIX), (HAR, FIX)])
def test_persistent_single_chain_bitwise(rk, gh, staged_refs, tiling, model, bc):
    y0, ref = staged_refs[(model, bc)]
    got = gh.gpu_run(y0, model=model, bc=bc, nsteps=37, kernel=rk.RK4_KERNEL_PERSISTENT, tiling=tiling)
    assert np.array_equal(got, ref)


def test_graph_replay_bitwise(rk, gh, staged_refs):
    y0, ref = staged_refs[(ROE, PER)]
    a = gh.gpu_run(y0, nsteps=37, tiling=(256, 4, 4), graphs=False)
    b = gh.gpu_run(y0, nsteps=37, tiling=(256, 4, 4), graphs=True)
    assert np.array_equal(a, ref) and np.array_equal(b, ref)


def test_split_integration_bitwise(rk, gh, staged_refs):
    """integrate(a) then integrate(b) equals integrate(a + b), bit for bit."""
    y0, ref = staged_refs[(ROE, FIX)]
    got = gh.gpu_run(y0, bc=FIX, nsteps=37, tiling=(128, 4, 4), chunks=[5, 1, 20, 11])
    assert np.array_equal(got, ref)


# ---- edge cases -----------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 33, 1000, 1017])
@pytest.mark.parametrize("bc", [PER, FIX])
def test_small_and_ragged_chains(rk, gh, n, bc):
    """Chains shorter than a halo, of one or two sites, and not a multiple of the tile."""
    y0 = ci.uniform_state(n, 3, seed=51 + n)
    ref = oracle.rk4_integrate(y0, ROE, bc, 0.01, 25)
    st = gh.gpu_run(y0, bc=bc, nsteps=25, kernel=rk.RK4_KERNEL_STAGED)
    for tiling in [(64, 1, 1), (256, 4, 4), (128, 2, 8)]:
        got = gh.gpu_run(y0, bc=bc, nsteps=25, tiling=tiling)
        assert np.array_equal(got, st), tiling
    assert rel(st, ref) <= 1e-12


def test_zero_and_odd_step_counts(rk, gh, staged_refs):
    y0, _ = staged_refs[(ROE, PER)]
    assert np.array_equal(gh.gpu_run(y0, nsteps=0), y0)
    for nsteps in (1, 3, 9, 17):
        ref = gh.gpu_run(y0, nsteps=nsteps, kernel=rk.RK4_KERNEL_STAGED)
        for t in [(256, 4, 1), (256, 4, 4), (256, 4, 8)]:
            assert np.array_equal(gh.gpu_run(y0, nsteps=nsteps, tiling=t), ref), (nsteps, t)


def test_reflection_and_shift_bitwise(rk, gh):
    y0 = ci.uniform_state(4099, 3, seed=61)
    base = gh.gpu_run(y0, nsteps=40, tiling=(256, 4, 4))
    shifted = gh.gpu_run(np.roll(y0, 517, axis=0), nsteps=40, tiling=(256, 4, 4))
    assert np.array_equal(shifted, np.roll(base, 517, axis=0))
    for bc in (PER, FIX):
        a = gh.gpu_run(y0, bc=bc, nsteps=40, tiling=(128, 8, 4))
        b = gh.gpu_run(np.ascontiguousarray(y0[::-1]), bc=bc, nsteps=40, tiling=(128, 8, 4))
        assert np.array_equal(a, b[::-1])


def test_dependency_cone_bitwise(rk, gh):
    """One perturbed site changes exactly the sites within 4 per step (Sec. 2.3's halo)."""
    n, site = 2000, 1000
    y0 = ci.uniform_state(n, 3, seed=71)
    y1 = y0.copy()
    y1[site, 0] += 0.5
    params = dict(kappa=20.0)
    for m in (1, 2, 3):
        a = gh.gpu_run(y0, bc=FIX, nsteps=m, dt=0.1, params=params, tiling=(128, 4, 2))
        b = gh.gpu_run(y1, bc=FIX, nsteps=m, dt=0.1, params=params, tiling=(128, 4, 2))
        changed = np.nonzero(np.any(a != b, axis=1))[0]
        assert changed.min() == site - 4 * m and changed.max() == site + 4 * m


# ---- batches ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_batch():
    lengths, kappa, bcs = ci.batch_spec(64, seed=81, nmin=1, nmax=3000)
    y0 = ci.uniform_state(int(lengths.sum()), 3, seed=82)
    return lengths, kappa, bcs, y0


def test_batch_vs_oracle_and_bitwise(rk, gh, small_batch):
    lengths, kappa, bcs, y0 = small_batch
    ref = oracle.batch_rk4_integrate(y0, lengths, kappa, bcs, nsteps=60)
    st = gh.gpu_run(y0, nsteps=60, lengths=lengths, kappas=kappa, bcs=bcs, kernel=rk.RK4_KERNEL_STAGED)
    assert rel(st, ref) <= 1e-12
    for kernel in (rk.RK4_KERNEL_BLOCKED, rk.RK4_KERNEL_PERSISTENT):
        for tiling in [(256, 4, 1), (128, 4, 4), (256, 8, 8)]:
            got = gh.gpu_run(y0, nsteps=60, lengths=lengths, kappas=kappa, bcs=bcs, kernel=kernel, tiling=tiling)
            assert np.array_equal(got, st), (kernel, tiling)


def test_batch_fp32_kahan_bitwise(rk, gh, small_batch):
    lengths, kappa, bcs, y0 = small_batch
    y32 = y0.astype(np.float32)
    st = gh.gpu_run(y32, precision=rk.RK4_FP32_KAHAN, nsteps=60, lengths=lengths, kappas=kappa, bcs=bcs,
                    kernel=rk.RK4_KERNEL_STAGED)
    got = gh.gpu_run(y32, precision=rk.RK4_FP32_KAHAN, nsteps=60, lengths=lengths, kappas=kappa, bcs=bcs,
                     tiling=(128, 4, 8))
    assert np.array_equal(got, st)


# ---- FP32 + Kahan ---------------------------------------------------------------------

def test_fp32_kahan_bitwise_and_error(rk, gh):
    """Blocked FP32-Kahan equals the staged FP32-Kahan kernel bit for bit; its error against the
    FP64 oracle (started from the same FP32 values) after 1000 steps is reported and bounded."""
    y0 = ci.uniform_state(65536, 3).astype(np.float32)
    st, c_st = gh.gpu_run(y0, precision=rk.RK4_FP32_KAHAN, nsteps=1000, kernel=rk.RK4_KERNEL_STAGED,
                          return_comp=True)
    # 1 and 2 sites per thread exchange neighbours by warp shuffles, 4 and 8 by per-thread
    # shared-memory slots; 2, 4 and 8 run on packed f32x2 instructions, 1 on scalar ones
    for tiling in [(256, 4, 4), (256, 8, 8), (512, 4, 16), (256, 1, 4), (128, 2, 8)]:
        got, c_got = gh.gpu_run(y0, precision=rk.RK4_FP32_KAHAN, nsteps=1000, tiling=tiling, return_comp=True)
        assert np.array_equal(got, st) and np.array_equal(c_got, c_st), tiling
    ref = oracle.rk4_integrate(y0.astype(np.float64), ROE, PER, 0.01, 1000)
    err = rel(st - c_st, ref)
    print(f"FP32-Kahan Roessler N=65536, 1000 steps: rel err vs FP64 oracle {err:.3e}")
    assert err <= FP32_KAHAN_TOL


def test_fp32_kahan_harmonic_error(rk, gh):
    y0 = ci.uniform_state(4096, 2).astype(np.float32)
    got, c = gh.gpu_run(y0, model=HAR, precision=rk.RK4_FP32_KAHAN, nsteps=1000, return_comp=True)
    ref = oracle.rk4_integrate(y0.astype(np.float64), HAR, PER, 0.01, 1000)
    err = rel(got - c, ref)
    print(f"FP32-Kahan harmonic N=4096, 1000 steps: rel err vs FP64 oracle {err:.3e}")
    assert err <= 1e-6


# ---- reductions, generator, status ----------------------------------------------------

def test_energy_matches_oracle_and_closed_form(rk, gh):
    import torch
    for bc in (PER, FIX):
        y0 = ci.uniform_state(100003, 2, seed=91 + bc)
        h = rk.rk4_chain_create(HAR, rk.RK4_FP64, y0.shape[0], 0.01, bc, dict(kappa=1.1, omega0=0.9))
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        st = gh.to_dev(y0, torch.float64)
        e = rk.rk4_chain_energy(h, st, None, ws)[0]
        ref = oracle.energy_harmonic(y0, bc, oracle.params(kappa=1.1, omega0=0.9))
        assert abs(e - ref) <= 1e-12 * abs(ref)
        modal = float(np.sum(cf.modal_energy(y0, bc, 1.1, 0.9)))
        assert abs(e - modal) <= 1e-11 * abs(modal)
        rk.rk4_chain_destroy(h)
    y0 = ci.uniform_state(77777, 3, seed=93)
    h = rk.rk4_chain_create(ROE, rk.RK4_FP64, y0.shape[0], 0.01, PER)
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    e = rk.rk4_chain_energy(h, gh.to_dev(y0, torch.float64), None, ws)[0]
    assert abs(e - oracle.half_norm2(y0)) <= 1e-12 * oracle.half_norm2(y0)
    rk.rk4_chain_destroy(h)


def test_energy_nonfinite_detected(rk, gh):
    import torch
    y0 = ci.uniform_state(5000, 3, seed=94)
    y0[1234, 1] = np.nan
    h = rk.rk4_chain_create(ROE, rk.RK4_FP64, y0.shape[0], 0.01, PER)
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    with pytest.raises(rk.RK4Error) as ei:
        rk.rk4_chain_energy(h, gh.to_dev(y0, torch.float64), None, ws)
    assert ei.value.code == rk.RK4_ENONFINITE
    rk.rk4_chain_destroy(h)


def test_batch_energy_per_chain(rk, gh, small_batch):
    import torch
    lengths, kappa, bcs, _ = small_batch
    y0 = ci.uniform_state(int(lengths.sum()), 2, seed=95)
    h = rk.rk4_batch_create(HAR, rk.RK4_FP64, lengths, kappa, bcs, 0.01)
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    e = rk.rk4_chain_energy(h, gh.to_dev(y0, torch.float64), None, ws)
    off = 0
    for c, n in enumerate(lengths):
        ref = oracle.energy_harmonic(y0[off:off + n], int(bcs[c]), oracle.params(kappa=float(kappa[c])))
        assert abs(e[c] - ref) <= 1e-12 * abs(ref)
        off += n
    rk.rk4_chain_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_fill_uniform_matches_host_generator(rk, prec):
    import torch
    count, start = 3 * 100003, 12345
    dtype = torch.float64 if prec == 0 else torch.float32
    out = torch.empty(count, dtype=dtype, device="cuda")
    rk.rk4_fill_uniform(out, count, ci.DEFAULT_SEED, start, prec)
    torch.cuda.synchronize()
    host = 2.0 * ci.uniform01(ci.DEFAULT_SEED, ci.STREAM_STATE, start, count) - 1.0
    host = host.astype(np.float64 if prec == 0 else np.float32)
    assert np.array_equal(out.cpu().numpy(), host)


def test_barrier_timeout_reports_status(rk, gh, small_batch):
    """The persistent kernel's grid barrier gives up after its bound and the host sees
    RK4_ETIMEOUT; the context stays usable afterwards."""
    import torch
    lengths, kappa, bcs, y0 = small_batch
    h = rk.rk4_batch_create(ROE, rk.RK4_FP64, lengths, kappa, bcs, 0.01)
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    st = gh.to_dev(y0, torch.float64)
    rk.rk4_debug_barrier_timeout(h, st, None, ws, 20_000_000)  # 20 ms
    assert rk.rk4_chain_status(h, ws) == rk.RK4_ETIMEOUT
    assert rk.rk4_chain_status(h, ws) == rk.RK4_OK  # status was cleared
    rk.rk4_chain_integrate(h, st, None, ws, 4)
    assert rk.rk4_chain_status(h, ws) == rk.RK4_OK
    rk.rk4_chain_destroy(h)


def test_abi_errors(rk):
    import torch
    h = rk.rk4_chain_create(ROE, rk.RK4_FP64, 1000, 0.01, PER)
    st = torch.zeros((1000, 3), dtype=torch.float64, device="cuda")
    need = rk.rk4_chain_workspace_bytes(h)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(rk.RK4Error) as ei:
        rk.rk4_chain_integrate(h, st, None, ws, 1, ws_bytes=need - 1)
    assert ei.value.code == rk.RK4_ENOMEM_WS
    with pytest.raises(rk.RK4Error) as ei:
        rk.rk4_chain_integrate(h, st, st, ws, 1)  # comp given to an FP64 handle
    assert ei.value.code == rk.RK4_EINVAL
    with pytest.raises(rk.RK4Error):
        rk.rk4_chain_integrate(h, st, None, ws, -1)
    rk.rk4_chain_destroy(h)


def test_time_bookkeeping(rk):
    import torch
    h = rk.rk4_chain_create(ROE, rk.RK4_FP64, 100, 0.01, PER)
    st = torch.zeros((100, 3), dtype=torch.float64, device="cuda")
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    rk.rk4_chain_set_time(h, 2.0)
    t = 0.0
    for _ in range(7):
        t = rk.rk4_chain_integrate(h, st, None, ws, 3)
    assert t == 2.0 + 21 * 0.01
    rk.rk4_chain_destroy(h)


@pytest.mark.parametrize("pinned", [True, False])
def test_integrate_host_buffers(rk, gh, pinned):
    """Host buffers in and out: page-locked memory moves by the library's copy kernel, pageable
    memory by cudaMemcpyAsync; an odd number of bytes leaves a tail the copy kernel moves
    singly (the harmonic chain of 20001 sites holds 320016 bytes, FP32-Kahan 160008)."""
    import torch
    for model, prec, n in ((ROE, rk.RK4_FP64, 20000), (HAR, rk.RK4_FP64, 20001), (ROE, rk.RK4_FP32_KAHAN, 20003)):
        D = 3 if model == ROE else 2
        fp32 = prec == rk.RK4_FP32_KAHAN
        y0 = ci.uniform_state(n, D, seed=97)
        if fp32:
            y0 = y0.astype(np.float32)
        ref, cref = gh.gpu_run(y0, model=model, precision=prec, nsteps=30, return_comp=True)
        h = rk.rk4_chain_create(model, prec, n, 0.01, PER)
        host = torch.from_numpy(y0.copy())
        hcomp = torch.zeros_like(host) if fp32 else None
        if pinned:
            host = host.pin_memory()
            hcomp = hcomp.pin_memory() if fp32 else None
        dev = torch.empty_like(host, device="cuda")
        dcomp = torch.empty_like(host, device="cuda") if fp32 else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_integrate_host(h, host, hcomp, dev, dcomp, ws, 30)
        assert np.array_equal(host.double().numpy(), ref), (model, prec)
        if fp32:
            assert np.array_equal(hcomp.double().numpy(), cref)
        rk.rk4_chain_destroy(h)


def test_batch_autotune_chooses_scheme_and_stays_bitwise(rk, gh, small_batch):
    """The autotuner may pick the persistent or the blocked scheme for a batch; either way the
    result is bit for bit the staged kernel's."""
    import torch
    lengths, kappa, bcs, y0 = small_batch
    ref = gh.gpu_run(y0, nsteps=60, lengths=lengths, kappas=kappa, bcs=bcs, kernel=rk.RK4_KERNEL_STAGED)
    h = rk.rk4_batch_create(ROE, rk.RK4_FP64, lengths, kappa, bcs, 0.01)
    st = gh.to_dev(y0, torch.float64)
    ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
    rk.rk4_chain_autotune(h, st.clone(), None, ws, 8)
    assert rk.rk4_chain_get_kernel(h) in (rk.RK4_KERNEL_PERSISTENT, rk.RK4_KERNEL_BLOCKED)
    rk.rk4_chain_integrate(h, st, None, ws, 60)
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy(), ref)
    rk.rk4_chain_destroy(h)


def test_checkpoint_resume_bitwise(rk, tmp_path):
    """integrate a steps, checkpoint, resume in a fresh handle, integrate b: bit-identical to
    a + b steps in one call, with the same clock (FP32-Kahan, so the compensation matters)."""
    import torch
    from paper_1412_0544_gb300 import checkpoint
    y0 = ci.uniform_state(30011, 3, seed=99).astype(np.float32)
    prec = rk.RK4_FP32_KAHAN

    def fresh():
        h = rk.rk4_chain_create(ROE, prec, y0.shape[0], 0.01, PER)
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        return h, ws

    h, ws = fresh()
    st = torch.from_numpy(y0).cuda()
    cp = torch.zeros_like(st)
    t_full = rk.rk4_chain_integrate(h, st, cp, ws, 70)
    full = (st.cpu().numpy(), cp.cpu().numpy())
    rk.rk4_chain_destroy(h)

    h, ws = fresh()
    st = torch.from_numpy(y0).cuda()
    cp = torch.zeros_like(st)
    rk.rk4_chain_integrate(h, st, cp, ws, 25)
    path = str(tmp_path / "chk.npz")
    checkpoint.save_handle(path, rk, h, st, cp, model="roessler")
    rk.rk4_chain_destroy(h)

    h, ws = fresh()
    st2, cp2, meta = checkpoint.restore_handle(path, rk, h)
    t_resumed = rk.rk4_chain_integrate(h, st2, cp2, ws, 45)
    rk.rk4_chain_destroy(h)
    assert meta["nstep"] == 25 and t_resumed == t_full
    assert np.array_equal(st2.cpu().numpy(), full[0]) and np.array_equal(cp2.cpu().numpy(), full[1])


def test_autotune_considers_staged_scheme_when_workspace_allows(rk, gh):
    """With a workspace large enough for the staged scheme, the autotuner also times it and keeps
    whichever scheme is faster; with the blocked scheme's workspace it keeps a tiled scheme.
    Either way the result equals the staged kernel's bit for bit."""
    import torch
    n, T = 1 << 20, 37
    y0 = ci.uniform_state(n, 3, seed=77)
    ref = gh.gpu_run(y0, nsteps=T, kernel=rk.RK4_KERNEL_STAGED)
    h = rk.rk4_chain_create(ROE, rk.RK4_FP64, n, 0.01, PER)
    try:
        small = rk.rk4_chain_workspace_bytes(h)
        rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_STAGED)
        large = rk.rk4_chain_workspace_bytes(h)
        rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_AUTO)
        assert large > small
        for nbytes, allowed in ((small, {rk.RK4_KERNEL_BLOCKED}),
                                (large, {rk.RK4_KERNEL_BLOCKED, rk.RK4_KERNEL_STAGED})):
            ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            st = gh.to_dev(y0, torch.float64)
            rk.rk4_chain_autotune(h, st.clone(), None, ws, 8)
            kern = rk.rk4_chain_get_kernel(h)
            assert kern in allowed, kern
            assert rk.rk4_chain_workspace_bytes(h) <= nbytes
            rk.rk4_chain_integrate(h, st, None, ws, T)
            assert np.array_equal(st.cpu().numpy(), ref), kern
            print(f"autotune with {nbytes} B of workspace: kernel {kern}")
            del ws, st
        rk.rk4_chain_set_tiling(h, 256, 4, 1)  # an explicit tiling returns to the tiled scheme
        assert rk.rk4_chain_get_kernel(h) == rk.RK4_KERNEL_BLOCKED
    finally:
        rk.rk4_chain_destroy(h)
