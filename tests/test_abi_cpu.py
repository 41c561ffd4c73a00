"""Host-side checks that need no GPU: the C-ABI library loads, exports every function the header
declares, and validates arguments before touching the device; plan logic; multi-rank helpers
over gloo (world size 2)."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1412_0544_gb300 as m
    return m


def test_library_exports_every_header_function(rk):
    names = rk.header_functions()
    assert len(names) >= 18
    lib = ctypes.CDLL(rk.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "rk4chain.h"\nint main(void){rk4_params p; rk4_params_default(&p); return 0;}\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c",
                        str(src), "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_argument_validation_without_gpu(rk):
    E = rk.RK4Error
    for bad in [dict(n=0), dict(dt=0.0), dict(dt=float("nan")), dict(bc=7), dict(model=5), dict(precision=3)]:
        kw = dict(model=0, precision=0, n=100, dt=0.01, bc=0)
        kw.update(bad)
        with pytest.raises(E) as ei:
            rk.rk4_chain_create(kw["model"], kw["precision"], kw["n"], kw["dt"], kw["bc"])
        assert ei.value.code == rk.RK4_EINVAL
    with pytest.raises(E):
        rk.rk4_batch_create(0, 0, [10, 0], [1.0, 1.0], [0, 0], 0.01)
    with pytest.raises(E):
        rk.rk4_batch_create(0, 0, [10, 5], [1.0, float("inf")], [0, 0], 0.01)
    with pytest.raises(E):
        rk.rk4_batch_create(0, 0, [10, 5], [1.0, 1.0], [0, 3], 0.01)
    with pytest.raises(E) as ei:  # an empty batch
        rk.rk4_batch_create(0, 0, [], [], [], 0.01)
    assert ei.value.code == rk.RK4_EINVAL


def test_tiling_rules(rk):
    h = rk.rk4_chain_create(0, 0, 1 << 20, 0.01, 0)
    try:
        t = rk.rk4_chain_get_tiling(h)
        assert t["G"] == t["block"] * t["v"] - 8 * t["k"]
        for bad in [(100, 4, 1), (256, 3, 1), (256, 4, 0), (256, 4, 17), (64, 1, 5), (2048, 1, 1)]:
            with pytest.raises(rk.RK4Error):
                rk.rk4_chain_set_tiling(h, *bad)
        rk.rk4_chain_set_tiling(h, 128, 8, 4)
        assert rk.rk4_chain_get_tiling(h) == {"block": 128, "v": 8, "k": 4, "G": 992}
        rk.rk4_chain_set_tiling(h, 0)
        assert rk.rk4_chain_get_tiling(h)["block"] == 256
    finally:
        rk.rk4_chain_destroy(h)


def test_workspace_sizes(rk):
    n = 1000
    h = rk.rk4_chain_create(0, 0, n, 0.01, 0)
    blocked = rk.rk4_chain_workspace_bytes(h)
    rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_STAGED)
    staged = rk.rk4_chain_workspace_bytes(h)
    rk.rk4_chain_destroy(h)
    assert blocked >= n * 3 * 8 and staged >= 3 * n * 3 * 8
    h = rk.rk4_chain_create(1, 1, n, 0.01, 1)
    assert rk.rk4_chain_workspace_bytes(h) >= 2 * n * 2 * 4  # state + compensation ping-pong
    rk.rk4_chain_destroy(h)


def test_null_buffers_rejected_before_launch(rk):
    h = rk.rk4_chain_create(0, 0, 100, 0.01, 0)
    with pytest.raises(rk.RK4Error) as ei:
        rk.rk4_chain_integrate(h, 0, None, 0, 1, ws_bytes=1 << 20)
    assert ei.value.code == rk.RK4_EINVAL
    with pytest.raises(rk.RK4Error) as ei:  # misaligned workspace
        rk.rk4_chain_integrate(h, 4096, None, 4096 + 8, 1, ws_bytes=1 << 20)
    assert ei.value.code == rk.RK4_EINVAL
    with pytest.raises(rk.RK4Error) as ei:  # too small
        rk.rk4_chain_integrate(h, 4096, None, 8192, 1, ws_bytes=16)
    assert ei.value.code == rk.RK4_ENOMEM_WS
    rk.rk4_chain_destroy(h)


def test_options(rk):
    h = rk.rk4_chain_create(0, 0, 100, 0.01, 0)
    rk.rk4_chain_set_option(h, rk.RK4_OPT_GRAPHS, 0)
    rk.rk4_chain_set_option(h, rk.RK4_OPT_TIMEOUT_NS, 10**8)
    with pytest.raises(rk.RK4Error):
        rk.rk4_chain_set_option(h, rk.RK4_OPT_GRAPHS, 2)
    with pytest.raises(rk.RK4Error):
        rk.rk4_chain_set_option(h, 99, 0)
    rk.rk4_chain_destroy(h)


def test_shard_chains_balances_and_partitions():
    from paper_1412_0544_gb300.dist import shard_chains
    import chain_inputs as ci
    lengths, _, _ = ci.batch_spec(4096)
    parts = [shard_chains(lengths, 4, r) for r in range(4)]
    allidx = sorted(i for p in parts for i in p)
    assert allidx == list(range(4096))
    loads = [int(lengths[p].sum()) for p in parts]
    assert max(loads) - min(loads) <= int(lengths.max())


_GLOO_WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
from paper_1412_0544_gb300 import dist as d
rank, world, local = d.init("gloo")
d.barrier()
m = d.max_over_ranks(1.0 + rank)
s = d.sum_over_ranks(10.0 * (rank + 1))
import chain_inputs as ci
lengths, _, _ = ci.batch_spec(256)
mine = d.shard_chains(lengths, world, rank)
print(json.dumps({"rank": rank, "max": m, "sum": s, "mine": mine}))
dist.destroy_process_group()
"""


def test_multirank_helpers_gloo(tmp_path):
    """Two CPU ranks: the barrier, the max-over-ranks timing reduction and the chain sharding."""
    script = tmp_path / "w.py"
    script.write_text(_GLOO_WORKER)
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT="29533", WORLD_SIZE="2")
    procs = []
    for r in range(2):
        e = dict(env, RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, str(script), ROOT], env=e, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(__import__("json").loads(o.strip().splitlines()[-1]))
    assert all(o["max"] == 2.0 and o["sum"] == 30.0 for o in outs)
    a, b = outs[0]["mine"], outs[1]["mine"]
    assert not set(a) & set(b) and sorted(a + b) == list(range(256))


def test_generic_scheme_validation(rk):
    h = rk.rk4_chain_create(0, 0, 1000, 0.01, 0)
    try:
        with pytest.raises(rk.RK4Error):  # not explicit: nonzero diagonal
            rk.rk4_chain_set_tableau(h, np.eye(2), np.array([0.5, 0.5]))
        with pytest.raises(rk.RK4Error):  # more than 7 stages
            rk.rk4_chain_set_tableau(h, np.zeros((8, 8)), np.full(8, 1 / 8))
        with pytest.raises(rk.RK4Error):
            rk.rk4_chain_set_coupling2(h, float("nan"))
        A = np.array([[0, 0, 0], [0.5, 0, 0], [-1.0, 2.0, 0]])
        rk.rk4_chain_set_tableau(h, A, np.array([1 / 6, 2 / 3, 1 / 6]))
        t = rk.rk4_chain_get_tiling(h)
        assert t["G"] == t["block"] * t["v"] - 2 * 3 * t["k"]  # halo = s * k per side
        rk.rk4_chain_set_coupling2(h, 0.5)
        t = rk.rk4_chain_get_tiling(h)
        assert t["G"] == t["block"] * t["v"] - 2 * 3 * 2 * t["k"]  # range 2 doubles it
        with pytest.raises(rk.RK4Error):  # generic kernels have 2 or 4 sites per thread
            rk.rk4_chain_set_tiling(h, 256, 1, 1)
        rk.rk4_chain_set_tiling(h, 128, 4, 3)
        assert rk.rk4_chain_get_tiling(h)["G"] == 512 - 2 * 18
        # Dormand-Prince 5: the seventh stage has weight 0 and feeds nothing, so the halo covers
        # the six stages the result needs
        import oracle_pins as P
        Ad, bd, _ = P.TABLEAUX["dopri5"]
        rk.rk4_chain_set_tableau(h, Ad, bd)
        rk.rk4_chain_set_tiling(h, 128, 4, 3)
        assert rk.rk4_chain_get_tiling(h)["G"] == 512 - 2 * 6 * 2 * 3
        rk.rk4_chain_set_tableau(h, A, np.array([1 / 6, 2 / 3, 1 / 6]))
        rk.rk4_chain_set_kernel(h, rk.RK4_KERNEL_STAGED)
        assert rk.rk4_chain_workspace_bytes(h) >= 4 * 1000 * 3 * 8  # stage state + 3 slopes
        rk.rk4_chain_set_tableau(h)  # back to classical RK4 (still range 2)
        rk.rk4_chain_set_coupling2(h, 0.0)
        assert rk.rk4_chain_get_tiling(h)["G"] == 256 * 4 - 8
    finally:
        rk.rk4_chain_destroy(h)


def test_site_params_validation(rk):
    h = rk.rk4_chain_create(0, 0, 1000, 0.01, 0)
    try:
        with pytest.raises(rk.RK4Error):  # device pointers must be 16-byte aligned
            rk.rk4_chain_set_site_params(h, 4096 + 8)
        rk.rk4_chain_set_site_params(h, 4096)
        assert rk.rk4_chain_get_tiling(h)["v"] in (2, 4)
        with pytest.raises(rk.RK4Error):  # heterogeneous kernels have 2 or 4 sites per thread
            rk.rk4_chain_set_tiling(h, 128, 8, 1)
        rk.rk4_chain_set_site_params(h, None)
        rk.rk4_chain_set_tiling(h, 128, 8, 1)
    finally:
        rk.rk4_chain_destroy(h)


def test_checkpoint_file_round_trip(rk, tmp_path):
    from paper_1412_0544_gb300 import checkpoint
    st = np.arange(30, dtype=np.float32).reshape(10, 3)
    cp = st * 1e-7
    p = str(tmp_path / "c.npz")
    checkpoint.save(p, st, cp, t0=1.5, nstep=42, model="roessler", n=10)
    s2, c2, meta = checkpoint.load(p)
    assert np.array_equal(s2, st) and np.array_equal(c2, cp)
    assert meta["t0"] == 1.5 and meta["nstep"] == 42 and meta["model"] == "roessler"
    h = rk.rk4_chain_create(0, 1, 10, 0.01, 0)
    rk.rk4_chain_set_clock(h, 1.5, 42)
    assert rk.rk4_chain_get_clock(h) == (1.5, 42)
    with pytest.raises(rk.RK4Error):
        rk.rk4_chain_set_clock(h, 0.0, -1)
    rk.rk4_chain_destroy(h)


def test_generic_halo_counts_needed_stages(rk):
    """The generic halo is (stages the result needs) x range x k: a stage with weight 0 that no
    needed stage uses cannot influence the step (host logic, no GPU)."""
    h = rk.rk4_chain_create(0, 0, 4000, 0.01, 0)
    try:
        def G_for(A, b, k=2):
            rk.rk4_chain_set_tableau(h, np.array(A, dtype=float), np.array(b, dtype=float))
            rk.rk4_chain_set_tiling(h, 128, 4, k)
            return rk.rk4_chain_get_tiling(h)["G"]
        # all three stages needed
        assert G_for([[0, 0, 0], [0.5, 0, 0], [-1, 2, 0]], [1 / 6, 2 / 3, 1 / 6]) == 512 - 2 * 3 * 2
        # only the first stage has weight and nothing uses the others: one stage
        assert G_for([[0, 0, 0], [0.5, 0, 0], [0, 1.0, 0]], [1.0, 0, 0]) == 512 - 2 * 1 * 2
        # the last stage uses the first only: stages 1 and 3 needed, the middle one dead
        assert G_for([[0, 0, 0], [0.5, 0, 0], [1.0, 0, 0]], [0, 0, 1.0]) == 512 - 2 * 2 * 2
        # a weightless stage that a needed stage uses is needed
        assert G_for([[0, 0, 0], [0.5, 0, 0], [0, 1.0, 0]], [0, 0, 1.0]) == 512 - 2 * 3 * 2
        rk.rk4_chain_set_coupling2(h, 0.3)  # range 2 doubles the halo
        assert G_for([[0, 0, 0], [0.5, 0, 0], [1.0, 0, 0]], [0, 0, 1.0]) == 512 - 2 * 2 * 2 * 2
    finally:
        rk.rk4_chain_destroy(h)
