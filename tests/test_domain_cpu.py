"""Sub-domain decomposition without a GPU: the library's domain layout and argument checks, the
decomposition itself run on the oracle (parts integrated as fixed-end chains with ghost zones,
swapped every floor(ghost / reach) steps, gathered bit-identical to the undivided chain), the
tightness of that bound, and the multi-rank form over gloo with two CPU ranks."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import chain_inputs as ci
import oracle
import oracle_pins as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PER, FIX = 0, 1


@pytest.fixture(scope="module")
def rk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1412_0544_gb300 as m
    return m


def layout(rk, model, n, bc, nparts, ghost, lengths=None):
    d = rk.rk4_domain_create(model, 0, n, 0.01, bc, nparts, ghost, part_lengths=lengths)
    try:
        return rk.rk4_domain_shape(d)[0], [rk.rk4_domain_part(d, p) for p in range(nparts)]
    finally:
        rk.rk4_domain_destroy(d)


def test_domain_layout(rk):
    rows, parts = layout(rk, 0, 1000, PER, 3, 8, [300, 500, 200])
    assert [p["sites"] for p in parts] == [300, 500, 200]
    assert [p["first_site"] for p in parts] == [0, 300, 800]
    assert all(p["ghost_left"] == p["ghost_right"] == 8 for p in parts)
    assert [p["row"] for p in parts] == [0, 316, 832] and rows == 1048
    rows, parts = layout(rk, 1, 1001, FIX, 4, 5)
    assert [p["sites"] for p in parts] == [251, 250, 250, 250]
    assert (parts[0]["ghost_left"], parts[-1]["ghost_right"]) == (0, 0)
    assert all(p["ghost_right"] == 5 for p in parts[:-1]) and all(p["ghost_left"] == 5 for p in parts[1:])
    assert rows == 1001 + 6 * 5
    rows, parts = layout(rk, 0, 77, FIX, 1, 0)  # one fixed-end part: no ghosts at all
    assert rows == 77 and parts[0]["ghost_left"] == parts[0]["ghost_right"] == 0
    rows, parts = layout(rk, 0, 77, PER, 1, 4)  # one periodic part is its own neighbour
    assert rows == 85


@pytest.mark.parametrize("bad", [
    dict(n=10, nparts=11), dict(nparts=0), dict(ghost=0), dict(ghost=-1), dict(lengths=[600, 300, 99]),
    dict(lengths=[10, 480, 510]), dict(bc=3), dict(model=7), dict(precision=2), dict(dt=0.0),
])
def test_domain_argument_validation(rk, bad):
    kw = dict(model=0, precision=0, n=1000, dt=0.01, bc=PER, nparts=3, ghost=16, lengths=None)
    kw.update(bad)
    with pytest.raises(rk.RK4Error) as ei:
        rk.rk4_domain_create(kw["model"], kw["precision"], kw["n"], kw["dt"], kw["bc"], kw["nparts"], kw["ghost"],
                             part_lengths=kw["lengths"])
    assert ei.value.code == rk.RK4_EINVAL


def decomposed(rk, y0, model, bc, nparts, ghost, nsteps, *, lengths=None, reach=4, tableau=None, prm=None,
               period=None, dt=0.01):
    """The decomposition on the oracle: the library's layout, ghost swaps by plain copies, every
    part integrated by the oracle as a fixed-end chain."""
    n = y0.shape[0]
    rows, parts = layout(rk, model, n, bc, nparts, ghost, lengths)
    dom = np.zeros((rows, y0.shape[1]))
    for p in parts:
        a = p["row"] + p["ghost_left"]
        dom[a:a + p["sites"]] = y0[p["first_site"]:p["first_site"] + p["sites"]]

    def swap():
        for i, p in enumerate(parts):
            if p["ghost_left"]:
                q = parts[(i - 1) % nparts]
                end = q["row"] + q["ghost_left"] + q["sites"]
                dom[p["row"]:p["row"] + ghost] = dom[end - ghost:end]
            if p["ghost_right"]:
                r = parts[(i + 1) % nparts]
                a = p["row"] + p["ghost_left"] + p["sites"]
                dom[a:a + ghost] = dom[r["row"] + r["ghost_left"]:r["row"] + r["ghost_left"] + ghost]

    if period is None:  # a single fixed-end part has no ghosts and runs in one go
        period = ghost // reach if any(p["ghost_left"] or p["ghost_right"] for p in parts) else max(nsteps, 1)
    done = 0
    while done < nsteps:
        m = min(period, nsteps - done)
        swap()
        for p in parts:
            a, b = p["row"], p["row"] + p["ghost_left"] + p["sites"] + p["ghost_right"]
            if tableau is None:
                dom[a:b] = oracle.rk4_integrate(dom[a:b], model, FIX, dt, m, prm)
            else:
                dom[a:b] = oracle.rk_integrate(dom[a:b], tableau[0], tableau[1], model, FIX, dt, m, prm)
        done += m
    out = np.empty_like(y0)
    for p in parts:
        a = p["row"] + p["ghost_left"]
        out[p["first_site"]:p["first_site"] + p["sites"]] = dom[a:a + p["sites"]]
    return out


CASES = [
    (0, PER, 3, 8, None), (0, FIX, 4, 12, None), (1, PER, 2, 4, [40, 1960]), (1, FIX, 5, 9, None),
    (0, PER, 1, 4, None), (0, FIX, 1, 0, None), (0, PER, 7, 5, [300, 250, 500, 5, 400, 300, 245]),
]


@pytest.mark.parametrize("model,bc,nparts,ghost,lengths", CASES)
def test_decomposition_on_oracle_bitwise(rk, model, bc, nparts, ghost, lengths):
    D = oracle.dim(model)
    y0 = ci.uniform_state(2000, D, seed=600 + nparts)
    ref = oracle.rk4_integrate(y0, model, bc, 0.01, 37)
    got = decomposed(rk, y0, model, bc, nparts, ghost, 37, lengths=lengths)
    assert np.array_equal(got, ref)


def test_decomposition_generic_scheme_on_oracle(rk):
    """Dormand-Prince 5 with second-neighbour coupling reaches at most 7 x 2 = 14 sites per step
    (12 counting only the stages the result needs); exchanging for 14 is safe either way."""
    A, b, _ = P.TABLEAUX["dopri5"]
    prm = oracle.params(kappa2=0.4)
    y0 = ci.uniform_state(1500, 3, seed=610)
    ref = oracle.rk_integrate(y0, A, b, 0, PER, 0.01, 11, prm)
    got = decomposed(rk, y0, 0, PER, 3, 30, 11, reach=14, tableau=(A, b), prm=prm)
    assert np.array_equal(got, ref)


def test_ghost_bound_is_tight(rk):
    """One step more between swaps than the ghost width allows lets the fixed ends' error reach
    the interiors (strong coupling and a large step, still inside RK4's stability region
    dt * 4 kappa = 2 < 2.78, make it visible above rounding)."""
    prm = oracle.params(kappa=5.0)
    y0 = ci.uniform_state(600, 3, seed=620)
    ref = oracle.rk4_integrate(y0, 0, PER, 0.1, 6, prm)
    ok = decomposed(rk, y0, 0, PER, 3, 8, 6, prm=prm, dt=0.1)
    bad = decomposed(rk, y0, 0, PER, 3, 8, 6, prm=prm, dt=0.1, period=3)
    assert np.array_equal(ok, ref)
    assert not np.array_equal(bad, ref)


_GLOO_DOMAIN = r"""
import json, sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np, torch, torch.distributed as dist
import chain_inputs as ci, oracle
import paper_1412_0544_gb300 as rk
from paper_1412_0544_gb300 import dist as d
rank, world, _ = d.init("gloo")
bc, ghost, n, nsteps, model = int(sys.argv[2]), 8, 1000, 29, int(sys.argv[3])
D = oracle.dim(model)
dom = rk.rk4_domain_create(model, 0, n, 0.01, bc, world, ghost)
part = rk.rk4_domain_part(dom, rank)
rk.rk4_domain_destroy(dom)
y0 = ci.uniform_state(n, D, seed=630)
ext = torch.zeros((part["ghost_left"] + part["sites"] + part["ghost_right"], D), dtype=torch.float64)
ext[part["ghost_left"]:part["ghost_left"] + part["sites"]] = torch.from_numpy(
    y0[part["first_site"]:part["first_site"] + part["sites"]])
def integrate(e, c, m):
    e.copy_(torch.from_numpy(oracle.rk4_integrate(e.numpy(), model, 1, 0.01, m)))
left, right = d.neighbours(rank, world, bc == 0)
exchange = d.exchange_ghosts_host if sys.argv[4] == "host" else d.exchange_ghosts
d.integrate_decomposed(ext, None, part, ghost, 4, nsteps, integrate, left, right, exchange=exchange)
mine = ext[part["ghost_left"]:part["ghost_left"] + part["sites"]].contiguous()
chunks = [torch.zeros_like(mine) for _ in range(world)]  # n splits evenly over the ranks
dist.all_gather(chunks, mine)
full = torch.cat(chunks)
ref = oracle.rk4_integrate(y0, model, bc, 0.01, nsteps)
print(json.dumps({"rank": rank, "equal": bool(np.array_equal(full.numpy(), ref))}))
dist.destroy_process_group()
"""


@pytest.mark.parametrize("bc,model,port,exchange", [(PER, 0, 29541, "direct"), (FIX, 1, 29542, "direct"),
                                                     (PER, 1, 29543, "host"), (FIX, 0, 29544, "host")])
def test_decomposition_two_gloo_ranks(tmp_path, bc, model, port, exchange):
    """One part per CPU rank, ghost zones swapped by point-to-point messages (directly, or
    through the edge-only host staging that device blocks use), parts integrated by the oracle:
    the gathered chain equals the undivided oracle run bit for bit."""
    script = tmp_path / "w.py"
    script.write_text(_GLOO_DOMAIN)
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2")
    procs = [subprocess.Popen([sys.executable, str(script), ROOT, str(bc), str(model), exchange],
                              env=dict(env, RANK=str(r), LOCAL_RANK=str(r)), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        o, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert all(o["equal"] for o in outs)
