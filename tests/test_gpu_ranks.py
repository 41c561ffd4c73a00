"""One chain split over two ranks, each integrating its part with the CUDA library.

Sec. 2.3's overlap applied to memory partitions across processes: every rank holds one part of
the chain with ghost zones (the rk4_domain_part layout), integrates it with
rk4_chain_integrate as a fixed-end chain of its block's length, and swaps ghost zones with its
neighbours every floor(ghost / 4) steps by point-to-point messages (gloo, through host memory:
only the block edges travel).  Both ranks run on the one GPU of the test; their kernels are
independent launches and never wait on each other (the ranks synchronise on the host between
integration periods).  The gathered chain must equal the undivided GPU run bit for bit and the
oracle within the parity tolerance.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK = r"""
import json, sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np, torch, torch.distributed as dist
import chain_inputs as ci, oracle
import paper_1412_0544_gb300 as rk
from paper_1412_0544_gb300 import dist as d
from tolerances import FP32_KAHAN_TOL
torch.cuda.set_device(0)
rank, world, _ = d.init("gloo")
bc, prec, model = int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4])
ghost, n, nsteps = 32, 40000, 203
D = oracle.dim(model)
fp32 = prec == rk.RK4_FP32_KAHAN
dtype = torch.float32 if fp32 else torch.float64
dom = rk.rk4_domain_create(model, prec, n, 0.01, bc, world, ghost)
part = rk.rk4_domain_part(dom, rank)
rk.rk4_domain_destroy(dom)
y0 = ci.uniform_state(n, D, seed=640 + bc)
if fp32:
    y0 = y0.astype(np.float32)
rows = part["ghost_left"] + part["sites"] + part["ghost_right"]
ext = torch.zeros((rows, D), dtype=dtype, device="cuda")
lo = part["ghost_left"]
ext[lo:lo + part["sites"]] = torch.from_numpy(y0[part["first_site"]:part["first_site"] + part["sites"]]).cuda()
comp = torch.zeros_like(ext) if fp32 else None
h = rk.rk4_chain_create(model, prec, rows, 0.01, rk.RK4_FIXED)  # the part as a fixed-end chain
ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
def integrate(e, c, m):
    rk.rk4_chain_integrate(h, e, c, ws, m)
left, right = d.neighbours(rank, world, bc == 0)
d.integrate_decomposed(ext, comp, part, ghost, 4, nsteps, integrate, left, right, exchange=d.exchange_ghosts_host)
torch.cuda.synchronize()
status = rk.rk4_chain_status(h, ws)
rk.rk4_chain_destroy(h)
mine = ext[lo:lo + part["sites"]].cpu().contiguous()
cmine = comp[lo:lo + part["sites"]].cpu().contiguous() if fp32 else torch.zeros(0)
chunks = [torch.zeros_like(mine) for _ in range(world)]  # n splits evenly over the ranks
dist.all_gather(chunks, mine)
cchunks = [torch.zeros_like(cmine) for _ in range(world)]
dist.all_gather(cchunks, cmine)
res = {"rank": rank, "status": status}
if rank == 0:
    full = torch.cat(chunks)
    # the undivided chain on the same GPU
    hw = rk.rk4_chain_create(model, prec, n, 0.01, bc)
    st = torch.from_numpy(y0).cuda()
    cp = torch.zeros_like(st) if fp32 else None
    wsw = torch.empty(rk.rk4_chain_workspace_bytes(hw), dtype=torch.uint8, device="cuda")
    rk.rk4_chain_integrate(hw, st, cp, wsw, nsteps)
    torch.cuda.synchronize()
    rk.rk4_chain_destroy(hw)
    res["bitwise_state"] = bool(torch.equal(full, st.cpu()))
    if fp32:
        res["bitwise_comp"] = bool(torch.equal(torch.cat(cchunks), cp.cpu()))
    ref = oracle.rk4_integrate(y0.astype(np.float64), model, bc, 0.01, nsteps)
    got = full.double().numpy() - (torch.cat(cchunks).double().numpy() if fp32 else 0.0)
    res["rel_err"] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    res["tol"] = FP32_KAHAN_TOL if fp32 else 1e-12
print(json.dumps(res))
dist.destroy_process_group()
"""


@pytest.mark.parametrize("bc,prec,model,port", [(0, 0, 0, 29551), (1, 0, 1, 29552), (0, 1, 0, 29553),
                                                (1, 1, 0, 29554)])
def test_two_ranks_each_integrating_on_the_gpu(tmp_path, bc, prec, model, port):
    script = tmp_path / "rank.py"
    script.write_text(_RANK)
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2")
    procs = [subprocess.Popen([sys.executable, str(script), ROOT, str(bc), str(prec), str(model)],
                              env=dict(env, RANK=str(r), LOCAL_RANK="0"), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        o, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert all(o["status"] == 0 for o in outs)
    r0 = next(o for o in outs if o["rank"] == 0)
    print(r0)
    assert r0["bitwise_state"] and r0.get("bitwise_comp", True)
    assert r0["rel_err"] <= r0["tol"]
