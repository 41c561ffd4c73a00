"""Cases run by both the release library and the bounds-checking debug library (see
test_gpu_debug_bounds.py): every scheme, ragged sizes, both precisions, reductions and the
sub-domain path.  run_all returns {case name: (arrays..., status code)}."""
import numpy as np

import chain_inputs as ci
import oracle_pins as P

PER, FIX = 0, 1


def _status(rk, h, ws):
    return rk.rk4_chain_status(h, ws)


def _single(rk, torch, *, model, prec, n, bc, nsteps, kernel=None, tiling=None, tableau=None, kappa2=0.0,
            site_params=False):
    D = 3 if model == 0 else 2
    dtype = torch.float32 if prec else torch.float64
    h = rk.rk4_chain_create(model, prec, n, 0.01, bc)
    try:
        if kernel is not None:
            rk.rk4_chain_set_kernel(h, kernel)
        if tableau is not None:
            rk.rk4_chain_set_tableau(h, *tableau)
        if kappa2:
            rk.rk4_chain_set_coupling2(h, kappa2)
        sp = None
        if site_params:
            sp = torch.from_numpy(P.het_params(n, model, 950 + n)).to(dtype).cuda()
            rk.rk4_chain_set_site_params(h, sp)
        if tiling is not None:
            rk.rk4_chain_set_tiling(h, *tiling)
        st = torch.from_numpy(ci.uniform_state(n, D, seed=951 + n)).to(dtype).cuda()
        cp = torch.zeros_like(st) if prec else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
        code = _status(rk, h, ws)
        e = rk.rk4_chain_energy(h, st, cp, ws) if not (site_params and model == 1) else np.zeros(1)
        out = [st.cpu().numpy(), e]
        if prec:
            out.append(cp.cpu().numpy())
        return out, code
    finally:
        rk.rk4_chain_destroy(h)


def _batch(rk, torch, *, prec, kernel, tiling, nsteps):
    lengths, kappa, bcs = ci.batch_spec(61, seed=960, nmin=1, nmax=1500)
    n = int(lengths.sum())
    dtype = torch.float32 if prec else torch.float64
    h = rk.rk4_batch_create(0, prec, lengths, kappa, bcs, 0.01)
    try:
        rk.rk4_chain_set_kernel(h, kernel)
        rk.rk4_chain_set_tiling(h, *tiling)
        st = torch.from_numpy(ci.uniform_state(n, 3, seed=961)).to(dtype).cuda()
        cp = torch.zeros_like(st) if prec else None
        ws = torch.empty(rk.rk4_chain_workspace_bytes(h), dtype=torch.uint8, device="cuda")
        rk.rk4_chain_integrate(h, st, cp, ws, nsteps)
        code = _status(rk, h, ws)
        e = rk.rk4_chain_energy(h, st, cp, ws)
        return [st.cpu().numpy(), e], code
    finally:
        rk.rk4_chain_destroy(h)


def _domain(rk, torch, *, prec, nsteps):
    n = 7001
    dtype = torch.float32 if prec else torch.float64
    d = rk.rk4_domain_create(0, prec, n, 0.01, FIX, 3, 12, part_lengths=[12, 4000, 2989])
    try:
        rows, D = rk.rk4_domain_shape(d)
        cst = torch.from_numpy(ci.uniform_state(n, D, seed=970)).to(dtype).cuda()
        ccp = torch.zeros_like(cst) if prec else None
        st = torch.zeros((rows, D), dtype=dtype, device="cuda")
        cp = torch.zeros_like(st) if prec else None
        ws = torch.empty(rk.rk4_domain_workspace_bytes(d), dtype=torch.uint8, device="cuda")
        rk.rk4_domain_scatter(d, cst, ccp, st, cp)
        rk.rk4_domain_integrate(d, st, cp, ws, nsteps)
        code = rk.rk4_domain_status(d, ws)
        e = rk.rk4_domain_energy(d, st, cp, ws)
        rk.rk4_domain_gather(d, st, cp, cst, ccp)
        return [cst.cpu().numpy(), np.array([e])], code
    finally:
        rk.rk4_domain_destroy(d)


def cases():
    dp = P.TABLEAUX["dopri5"]
    c = {}
    for prec in (0, 1):
        for model, bc, n in [(0, PER, 5003), (0, FIX, 3), (1, FIX, 1025), (1, PER, 1)]:
            tag = f"p{prec}_m{model}_bc{bc}_n{n}"
            c[f"staged_{tag}"] = lambda rk, torch, a=dict(model=model, prec=prec, n=n, bc=bc): _single(
                rk, torch, nsteps=9, kernel=1, **a)
            for t in [(64, 1, 1), (256, 4, 2), (128, 8, 16), (512, 2, 3)]:
                c[f"blocked_{tag}_{t}"] = lambda rk, torch, a=dict(model=model, prec=prec, n=n, bc=bc), t=t: _single(
                    rk, torch, nsteps=2 * t[2] + 1, kernel=2, tiling=t, **a)
            c[f"persistent_{tag}"] = lambda rk, torch, a=dict(model=model, prec=prec, n=n, bc=bc): _single(
                rk, torch, nsteps=11, kernel=3, tiling=(128, 4, 2), **a)
        c[f"generic_staged_p{prec}"] = lambda rk, torch, p=prec: _single(
            rk, torch, model=0, prec=p, n=2003, bc=PER, nsteps=5, kernel=1, tableau=dp[:2], kappa2=0.3)
        c[f"generic_blocked_p{prec}"] = lambda rk, torch, p=prec: _single(
            rk, torch, model=1, prec=p, n=2003, bc=FIX, nsteps=5, kernel=2, tiling=(128, 4, 2), tableau=dp[:2],
            kappa2=0.3)
        c[f"het_blocked_p{prec}"] = lambda rk, torch, p=prec: _single(
            rk, torch, model=0, prec=p, n=3001, bc=FIX, nsteps=7, kernel=2, tiling=(256, 2, 3), site_params=True)
        c[f"het_staged_p{prec}"] = lambda rk, torch, p=prec: _single(
            rk, torch, model=1, prec=p, n=3001, bc=PER, nsteps=7, kernel=1, site_params=True)
        c[f"batch_persistent_p{prec}"] = lambda rk, torch, p=prec: _batch(rk, torch, prec=p, kernel=3,
                                                                           tiling=(128, 4, 4), nsteps=9)
        c[f"batch_blocked_p{prec}"] = lambda rk, torch, p=prec: _batch(rk, torch, prec=p, kernel=2,
                                                                        tiling=(256, 4, 2), nsteps=9)
        # packed batch tiles with one, two and eight sites per thread (segment windows start
        # at multiples of v slots, so shared-memory tile offsets of every alignment occur)
        for t, kern in (((256, 1, 2), 2), ((128, 2, 3), 3), ((128, 8, 4), 2)):
            c[f"batch_packed_{kern}_{t}_p{prec}"] = lambda rk, torch, p=prec, t=t, kern=kern: _batch(
                rk, torch, prec=p, kernel=kern, tiling=t, nsteps=2 * t[2] + 1)
        c[f"batch_staged_p{prec}"] = lambda rk, torch, p=prec: _batch(rk, torch, prec=p, kernel=1,
                                                                       tiling=(256, 4, 2), nsteps=3)
        c[f"domain_p{prec}"] = lambda rk, torch, p=prec: _domain(rk, torch, prec=p, nsteps=13)
    return c


def run_all(rk, torch):
    return {name: fn(rk, torch) for name, fn in cases().items()}
