"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each ``pin_*`` function takes an oracle library handle and returns ``(ok, detail)``.  The
ordinary tests assert every pin holds for the real oracle; the mutation test rebuilds the
oracle with one planted mistake at a time and asserts that some pin fails.  Nothing here
reuses the oracle's arithmetic: references are normal-mode closed forms, a library ODE
integrator (scipy's DOP853) on the paper's equations written as whole-array numpy, an
arbitrary-precision brute force, fixed points, and exact invariants.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp

import chain_inputs as ci
import oracle
import closed_form as cf

PER, FIX = oracle.PERIODIC, oracle.FIXED
ROE, HAR = oracle.ROESSLER, oracle.HARMONIC


# ---- harmonic chain: closed forms ------------------------------------------------------

def pin_harmonic_modal(lib, n=64, bc=PER, nsteps=1000, dt=0.01, kappa=1.3, omega0=0.7, tol=1e-12):
    """RK4 on the harmonic chain equals R^n applied per normal mode (exact up to rounding)."""
    y0 = ci.uniform_state(n, 2, seed=1000 + n + 7 * bc)
    prm = oracle.params(kappa=kappa, omega0=omega0)
    got = oracle.rk4_integrate(y0, HAR, bc, dt, nsteps, prm, lib=lib)
    ref = cf.rk4_modal(y0, bc, kappa, omega0, dt, nsteps)
    err = cf.rel_inf(got, ref)
    return err < tol, f"harmonic modal n={n} bc={bc}: rel err {err:.3e} (tol {tol:g})"


def pin_harmonic_order4(lib, n=32, bc=PER, T=2.0, kappa=1.0, omega0=1.0):
    """Error against the exact flow shrinks 16x per halving of dt (fourth order)."""
    y0 = ci.uniform_state(n, 2, seed=2000 + n + bc)
    prm = oracle.params(kappa=kappa, omega0=omega0)
    exact = cf.exact_flow(y0, bc, kappa, omega0, T)
    errs = []
    for dt in (0.05, 0.025, 0.0125):
        got = oracle.rk4_integrate(y0, HAR, bc, dt, int(round(T / dt)), prm, lib=lib)
        errs.append(cf.rel_inf(got, exact))
    orders = [float(np.log2(errs[i] / errs[i + 1])) for i in range(2)]
    ok = all(3.85 < p < 4.2 for p in orders)
    return ok, f"harmonic order bc={bc}: errors {errs}, observed orders {orders}"


def pin_harmonic_energy(lib, n=48, bc=PER, nsteps=1000, dt=0.05, kappa=1.1, omega0=0.9, tol=1e-12):
    """Energy of the initial state equals the modal sum, and after n steps equals
    sum_m E_m(0) rho(h_m)^n (RK4's exact per-mode energy factor)."""
    y0 = ci.uniform_state(n, 2, seed=3000 + n + bc)
    prm = oracle.params(kappa=kappa, omega0=omega0)
    e0 = oracle.energy_harmonic(y0, bc, prm, lib=lib)
    e0_ref = float(np.sum(cf.modal_energy(y0, bc, kappa, omega0)))
    y = oracle.rk4_integrate(y0, HAR, bc, dt, nsteps, prm, lib=lib)
    e1 = oracle.energy_harmonic(y, bc, prm, lib=lib)
    e1_ref = cf.rk4_energy(y0, bc, kappa, omega0, dt, nsteps)
    r0 = abs(e0 - e0_ref) / e0_ref
    r1 = abs(e1 - e1_ref) / e1_ref
    drift = abs(e1_ref - e0_ref) / e0_ref
    ok = r0 < tol and r1 < tol and drift > 100 * tol  # the drift itself must be resolved
    return ok, f"energy bc={bc}: E0 rel {r0:.2e}, En rel {r1:.2e}, modal drift {drift:.2e}"


# ---- Roessler chain: fixed points, library integrator, special cases ----------------

def roessler_fixed_points(a=0.2, b=1.0, c=9.0):
    """Equilibria of Eq. (6): y = -z, x = a z, a z^2 - c z + b = 0."""
    disc = np.sqrt(c * c - 4 * a * b)
    out = []
    for z in ((c - disc) / (2 * a), (c + disc) / (2 * a)):
        out.append(np.array([a * z, -z, z]))
    return out


def pin_roessler_fixed_point(lib, n=16, nsteps=1000, dt=0.01, tol=1e-12):
    """A uniform periodic chain sitting at an equilibrium of Eq. (6) stays there."""
    worst = 0.0
    for fp in roessler_fixed_points():
        y0 = np.tile(fp, (n, 1))
        got = oracle.rk4_integrate(y0, ROE, PER, dt, nsteps, lib=lib)
        worst = max(worst, cf.rel_inf(got, y0))
    return worst < tol, f"Roessler equilibria drift {worst:.2e}"


def roessler_chain_rhs(bc, kappa, a=0.2, b=1.0, c=9.0, kappa2=0.0):
    """Eq. (2) with f, g of Eqs. (6)-(7) as whole-array numpy (for scipy's integrator), plus an
    optional second-neighbour coupling kappa2."""
    def shifted(x, s):  # x_{i+s}, zero beyond fixed ends
        if bc == PER:
            return np.roll(x, -s)
        out = np.zeros_like(x)
        if s > 0:
            out[:-s] = x[s:]
        else:
            out[-s:] = x[:s]
        return out

    def F(_t, v):
        r = v.reshape(-1, 3)
        x, y, z = r[:, 0], r[:, 1], r[:, 2]
        xl, xr = shifted(x, -1), shifted(x, 1)
        xl2, xr2 = shifted(x, -2), shifted(x, 2)
        out = np.empty_like(r)
        out[:, 0] = -y - z + kappa * (xl - 2 * x + xr) + kappa2 * (xl2 - 2 * x + xr2)
        out[:, 1] = x + a * y
        out[:, 2] = b + z * (x - c)
        return out.reshape(-1)
    return F


def pin_roessler_vs_dop853(lib, n=6, bc=PER, kappa=1.0, T=0.5, kappa2=0.0):
    """RK4 converges at fourth order to scipy's DOP853 solution of the paper's equations."""
    y0 = ci.uniform_state(n, 3, seed=4000 + n + bc)
    sol = solve_ivp(roessler_chain_rhs(bc, kappa, kappa2=kappa2), (0.0, T), y0.reshape(-1), method="DOP853",
                    rtol=1e-13, atol=1e-13)
    ref = sol.y[:, -1].reshape(-1, 3)
    prm = oracle.params(kappa=kappa, kappa2=kappa2)
    errs = []
    for dt in (0.025, 0.0125, 0.00625):
        got = oracle.rk4_integrate(y0, ROE, bc, dt, int(round(T / dt)), prm, lib=lib)
        errs.append(cf.rel_inf(got, ref))
    orders = [float(np.log2(errs[i] / errs[i + 1])) for i in range(2)]
    ok = all(3.85 < p < 4.25 for p in orders) and errs[-1] < 1e-7
    return ok, f"Roessler vs DOP853 bc={bc}: errors {errs}, observed orders {orders}"


def pin_roessler_uniform_single(lib, n=5, nsteps=300, dt=0.01):
    """A uniform chain has zero coupling (Eq. (7) vanishes), so every site follows the
    single-oscillator trajectory bit for bit; that trajectory converges to DOP853's."""
    r0 = ci.uniform_state(1, 3, seed=5000)[0]
    y0 = np.tile(r0, (n, 1))
    got = oracle.rk4_integrate(y0, ROE, PER, dt, nsteps, lib=lib)
    same = bool(np.all(got == got[0]))
    T = nsteps * dt
    sol = solve_ivp(roessler_chain_rhs(PER, 0.0), (0.0, T), r0, method="DOP853", rtol=1e-13, atol=1e-13)
    err = cf.rel_inf(got[0], sol.y[:, -1])
    return same and err < 1e-7, f"uniform chain: sites identical={same}, err vs DOP853 {err:.2e}"


def pin_roessler_decoupled(lib, n=5, nsteps=200, dt=0.01):
    """kappa = 0 decouples the sites: each equals a one-site periodic chain, bit for bit."""
    y0 = ci.uniform_state(n, 3, seed=6000)
    prm = oracle.params(kappa=0.0)
    got = oracle.rk4_integrate(y0, ROE, PER, dt, nsteps, prm, lib=lib)
    ok = True
    for i in range(n):
        one = oracle.rk4_integrate(y0[i:i + 1], ROE, PER, dt, nsteps, prm, lib=lib)
        ok &= bool(np.array_equal(one[0], got[i]))
    return ok, f"kappa=0 decoupling bitwise={ok}"


# ---- brute force in arbitrary precision ------------------------------------------------

def brute_force_rk4(y0, model, bc, prm, dt, nsteps, dps=40):
    """Classical RK4 as a dense vector map in mpmath, neighbours from explicit lists."""
    import mpmath as mp
    mp.mp.dps = dps
    a, b, c, kappa, omega0, kappa2 = (mp.mpf(float(v)) for v in prm)
    y = [[mp.mpf(float(v)) for v in row] for row in np.asarray(y0)]
    n = len(y)

    def at(i):  # explicit neighbour lists: an index, or None for a fixed-end ghost
        if bc == PER:
            return i % n
        return i if 0 <= i < n else None

    nb = [(at(i - 1), at(i + 1), at(i - 2), at(i + 2)) for i in range(n)]
    h = mp.mpf(float(dt))

    def F(state):
        out = []
        for i, idx in enumerate(nb):
            xl, xr, xl2, xr2 = (state[j][0] if j is not None else mp.mpf(0) for j in idx)
            s = state[i]
            g = kappa * (xl + xr - 2 * s[0]) + kappa2 * (xl2 + xr2 - 2 * s[0])
            if model == ROE:
                out.append([-s[1] - s[2] + g, s[0] + a * s[1], b + s[2] * (s[0] - c)])
            else:
                out.append([s[1], -omega0 ** 2 * s[0] + g])
        return out

    def axpy(u, alpha, v):
        return [[ui + alpha * vi for ui, vi in zip(ur, vr)] for ur, vr in zip(u, v)]

    for _ in range(nsteps):
        k1 = F(y)
        k2 = F(axpy(y, h / 2, k1))
        k3 = F(axpy(y, h / 2, k2))
        k4 = F(axpy(y, h, k3))
        y = [[yi + h / 6 * (p + 2 * q + 2 * r + s) for yi, p, q, r, s in zip(*rows)]
             for rows in zip(y, k1, k2, k3, k4)]
    return np.array([[float(v) for v in row] for row in y])


def pin_brute_force(lib, n=4, model=ROE, bc=PER, nsteps=100, dt=0.01, tol=1e-13, kappa2=0.0):
    D = oracle.dim(model)
    y0 = ci.uniform_state(n, D, seed=7000 + n + 10 * model + bc)
    prm = oracle.params(kappa=1.25, omega0=0.8, kappa2=kappa2)
    got = oracle.rk4_integrate(y0, model, bc, dt, nsteps, prm, lib=lib)
    ref = brute_force_rk4(y0, model, bc, prm, dt, nsteps)
    err = cf.rel_inf(got, ref)
    return err < tol, f"brute force n={n} model={model} bc={bc}: rel err {err:.2e}"


# ---- exact invariants -------------------------------------------------------------------

def pin_shift_invariance(lib, n=40, shift=7, nsteps=50):
    """Periodic chain: integrating a cyclically shifted state gives the shifted result,
    bit for bit (every site runs the same operations)."""
    y0 = ci.uniform_state(n, 3, seed=8000)
    a = oracle.rk4_integrate(np.roll(y0, shift, axis=0), ROE, PER, 0.01, nsteps, lib=lib)
    b = np.roll(oracle.rk4_integrate(y0, ROE, PER, 0.01, nsteps, lib=lib), shift, axis=0)
    ok = bool(np.array_equal(a, b))
    return ok, f"shift invariance bitwise={ok}"


def pin_reflection(lib, n=33, nsteps=100, tol=1e-12):
    """Reflection i -> N+1-i maps solutions to solutions (to rounding: the oracle's
    Laplacian adds its neighbours in a fixed left-right order)."""
    worst = 0.0
    for bc in (PER, FIX):
        y0 = ci.uniform_state(n, 3, seed=8100 + bc)
        a = oracle.rk4_integrate(y0[::-1], ROE, bc, 0.01, nsteps, lib=lib)[::-1]
        b = oracle.rk4_integrate(y0, ROE, bc, 0.01, nsteps, lib=lib)
        worst = max(worst, cf.rel_inf(a, b))
    return worst < tol, f"reflection max rel err {worst:.2e}"


def pin_dependency_cone(lib, n=64, site=24):
    """Perturbing one site changes, after m steps, exactly the sites within 4m of it: each
    of the four stages re-evaluates the coupling (the paper's halo of s sites per step,
    Sec. 2.3).  A strong coupling and a large step keep the influence at distance 4m above
    the rounding level, so the cone's edge is visible."""
    y0 = ci.uniform_state(n, 3, seed=8200)
    y1 = y0.copy()
    y1[site, 0] += 0.5
    prm = oracle.params(kappa=20.0)
    ok = True
    detail = []
    for m in (1, 2, 3):
        a = oracle.rk4_integrate(y0, ROE, FIX, 0.1, m, prm, lib=lib)
        b = oracle.rk4_integrate(y1, ROE, FIX, 0.1, m, prm, lib=lib)
        changed = np.nonzero(np.any(a != b, axis=1))[0]
        lo, hi = int(changed.min()), int(changed.max())
        detail.append((m, lo, hi))
        ok &= (lo == site - 4 * m) and (hi == site + 4 * m)
    return ok, f"dependency cone (m, lo, hi) = {detail}"


# ---- general explicit tableaux (the technique applies to any explicit RK, Sec. 2) -----

TABLEAUX = {
    # name: (A, b, order)
    "euler": (np.array([[0.0]]), np.array([1.0]), 1),
    "heun2": (np.array([[0, 0], [1.0, 0]]), np.array([0.5, 0.5]), 2),
    "kutta3": (np.array([[0, 0, 0], [0.5, 0, 0], [-1.0, 2.0, 0]]), np.array([1 / 6, 2 / 3, 1 / 6]), 3),
    "rk4": (oracle.RK4_A, oracle.RK4_B, 4),
    "rule38": (np.array([[0, 0, 0, 0], [1 / 3, 0, 0, 0], [-1 / 3, 1.0, 0, 0], [1.0, -1.0, 1.0, 0]]),
               np.array([1 / 8, 3 / 8, 3 / 8, 1 / 8]), 4),
    # Dormand and Prince (1980), the fifth-order solution of RK5(4)7M used with a fixed step
    "dopri5": (np.array([
        [0, 0, 0, 0, 0, 0, 0],
        [1 / 5, 0, 0, 0, 0, 0, 0],
        [3 / 40, 9 / 40, 0, 0, 0, 0, 0],
        [44 / 45, -56 / 15, 32 / 9, 0, 0, 0, 0],
        [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729, 0, 0, 0],
        [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656, 0, 0],
        [35 / 384, 0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0]]),
        np.array([35 / 384, 0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0]), 5),
}


def pin_tableau_orders(lib, n=16, T=1.0):
    """Each tableau's error against the exact harmonic flow falls as dt^order."""
    y0 = ci.uniform_state(n, 2, seed=9000)
    exact = cf.exact_flow(y0, PER, 1.0, 1.0, T)
    detail = {}
    ok = True
    for name, (A, b, order) in TABLEAUX.items():
        errs = []
        for dt in ((0.2, 0.1) if order >= 5 else (0.05, 0.025)):
            got = oracle.rk_integrate(y0, A, b, HAR, PER, dt, int(round(T / dt)), lib=lib)
            errs.append(cf.rel_inf(got, exact))
        p = np.log2(errs[0] / errs[1])
        detail[name] = round(float(p), 3)
        ok &= abs(p - order) < 0.2
    return ok, f"observed orders {detail}"


# ---- next-nearest-neighbour coupling (the longer coupling range of Sec. 5) --------------

def pin_nnn_modal(lib, n=48, nsteps=800, dt=0.01, kappa=1.1, kappa2=0.6, omega0=0.8, tol=1e-12):
    """Periodic harmonic chain with second-neighbour coupling: Fourier modes still diagonalise
    it, omega_m^2 = omega0^2 + 4 kappa sin^2(pi m/N) + 4 kappa2 sin^2(2 pi m/N)."""
    y0 = ci.uniform_state(n, 2, seed=9100 + n)
    prm = oracle.params(kappa=kappa, omega0=omega0, kappa2=kappa2)
    got = oracle.rk4_integrate(y0, HAR, PER, dt, nsteps, prm, lib=lib)
    ref = cf.rk4_modal(y0, PER, kappa, omega0, dt, nsteps, kappa2=kappa2)
    e0 = oracle.energy_harmonic(y0, PER, prm, lib=lib)
    e0_ref = float(np.sum(cf.modal_energy(y0, PER, kappa, omega0, kappa2=kappa2)))
    err = cf.rel_inf(got, ref)
    ok = err < tol and abs(e0 - e0_ref) < tol * e0_ref
    return ok, f"NNN harmonic modal: rel err {err:.2e}, energy rel {abs(e0 - e0_ref) / e0_ref:.2e}"


def pin_nnn_energy_fixed(lib, n=12, nsteps=400, dt=0.02):
    """Fixed ends with second-neighbour bonds: the energy (ghost bonds included) is conserved
    by the exact flow, so RK4's drift is O(dt^4) per unit time and shrinks ~2^4 per halving."""
    y0 = ci.uniform_state(n, 2, seed=9200)
    prm = oracle.params(kappa=1.0, omega0=1.0, kappa2=0.7)
    e0 = oracle.energy_harmonic(y0, FIX, prm, lib=lib)
    drifts = []
    for k in range(3):
        h = dt / 2 ** k
        y = oracle.rk4_integrate(y0, HAR, FIX, h, nsteps * 2 ** k, prm, lib=lib)
        drifts.append(abs(oracle.energy_harmonic(y, FIX, prm, lib=lib) - e0) / e0)
    orders = [float(np.log2(drifts[i] / drifts[i + 1])) for i in range(2)]
    ok = all(3.5 < p < 6.5 for p in orders)
    return ok, f"NNN fixed-end energy drift {drifts}, orders {orders}"


def pin_nnn_cone(lib, n=96, site=48):
    """With second neighbours the influence of one site spreads exactly 2 sites per stage, 8 per
    step (twice the overlap, as Sec. 5 says for next-nearest coupling)."""
    y0 = ci.uniform_state(n, 3, seed=9300)
    y1 = y0.copy()
    y1[site, 0] += 0.5
    prm = oracle.params(kappa=5.0, kappa2=10.0)
    detail, ok = [], True
    for m in (1, 2):
        a = oracle.rk4_integrate(y0, ROE, FIX, 0.1, m, prm, lib=lib)
        b = oracle.rk4_integrate(y1, ROE, FIX, 0.1, m, prm, lib=lib)
        changed = np.nonzero(np.any(a != b, axis=1))[0]
        detail.append((m, int(changed.min()), int(changed.max())))
        ok &= changed.min() == site - 8 * m and changed.max() == site + 8 * m
    return ok, f"NNN cone {detail}"


def pin_dopri5_nnn_cone(lib, n=160, site=80):
    """Dormand-Prince 5 with second neighbours: the seventh stage has weight 0 and no stage uses
    it, so one step's influence spreads through the six stages the result needs, exactly 2 x 6
    = 12 sites per step (not 14) -- the halo and sub-domain reach the GPU path sizes by."""
    A, b, _ = TABLEAUX["dopri5"]
    y0 = ci.uniform_state(n, 3, seed=9310)
    y1 = y0.copy()
    y1[site, 0] += 0.5
    prm = oracle.params(kappa=5.0, kappa2=10.0)
    detail, ok = [], True
    for m in (1, 2, 3):
        a = oracle.rk_integrate(y0, A, b, ROE, FIX, 0.05, m, prm, lib=lib)
        c = oracle.rk_integrate(y1, A, b, ROE, FIX, 0.05, m, prm, lib=lib)
        changed = np.nonzero(np.any(a != c, axis=1))[0]
        detail.append((m, int(changed.min()), int(changed.max())))
        ok &= changed.min() == site - 12 * m and changed.max() == site + 12 * m
    return ok, f"Dormand-Prince 5 + NNN cone {detail}"


# ---- heterogeneous chains, Eq. (1): site-dependent f_i and g_i ---------------------------

def het_params(n, model, seed, kappa_scale=1.0):
    """Seeded per-site parameters spread around the paper's values."""
    u = ci.uniform01(seed, 9, 0, 4 * n).reshape(n, 4)
    if model == ROE:
        return np.stack([0.15 + 0.1 * u[:, 0], 0.8 + 0.4 * u[:, 1], 8.0 + 2.0 * u[:, 2],
                         kappa_scale * (0.5 + 1.5 * u[:, 3])], axis=1)
    return np.stack([0.5 + u[:, 0], kappa_scale * (0.5 + 1.5 * u[:, 1])], axis=1)


def pin_het_decoupled(lib, n=7, nsteps=200):
    """kappa_i = 0: every site is its own oscillator with its own (a_i, b_i, c_i), equal bit for
    bit to a one-site run of the (pinned) homogeneous integrator with those parameters."""
    y0 = ci.uniform_state(n, 3, seed=9400)
    sp = het_params(n, ROE, 9401, kappa_scale=0.0)
    got = oracle.rk4_integrate_het(y0, sp, ROE, PER, 0.01, nsteps, lib=lib)
    ok = True
    for i in range(n):
        prm = oracle.params(a=sp[i, 0], b=sp[i, 1], c=sp[i, 2], kappa=0.0)
        one = oracle.rk4_integrate(y0[i:i + 1], ROE, PER, 0.01, nsteps, prm, lib=lib)
        ok &= bool(np.array_equal(one[0], got[i]))
    return ok, f"heterogeneous decoupled sites bitwise={ok}"


def pin_het_harmonic_eigen(lib, n=40, nsteps=600, dt=0.01, kappa=1.3):
    """Harmonic chain with site-dependent omega_i and uniform kappa: K = diag(omega_i^2) - kappa L
    is symmetric, so its eigenvectors (numpy eigh) diagonalise the system and RK4 acts on each
    eigenmode as R^n (the closed form of the homogeneous chain, per eigenvalue)."""
    y0 = ci.uniform_state(n, 2, seed=9500)
    sp = het_params(n, HAR, 9501)
    sp[:, 1] = kappa
    worst = 0.0
    for bc in (PER, FIX):
        L = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
        if bc == PER:
            L[0, -1] += 1.0
            L[-1, 0] += 1.0
        K = np.diag(sp[:, 0]) - kappa * L
        lam, V = np.linalg.eigh(K)
        w = np.sqrt(lam)
        h = w * dt
        alpha, beta = 1 - h ** 2 / 2 + h ** 4 / 24, 1 - h ** 2 / 6
        rho, theta = alpha ** 2 + (beta * h) ** 2, np.arctan2(beta * h, alpha)
        qh, sh = V.T @ y0[:, 0], (V.T @ y0[:, 1]) / w
        amp, ang = rho ** (nsteps / 2), nsteps * theta
        q1 = amp * (np.cos(ang) * qh + np.sin(ang) * sh)
        s1 = amp * (-np.sin(ang) * qh + np.cos(ang) * sh)
        ref = np.stack([V @ q1, V @ (s1 * w)], axis=1)
        got = oracle.rk4_integrate_het(y0, sp, HAR, bc, dt, nsteps, lib=lib)
        worst = max(worst, cf.rel_inf(got, ref))
    return worst < 1e-12, f"heterogeneous harmonic vs eigen-decomposition rel err {worst:.2e}"


def pin_het_roessler_dop853(lib, n=6, T=0.5):
    """Site-dependent Roessler parameters and couplings: fourth-order convergence to DOP853."""
    y0 = ci.uniform_state(n, 3, seed=9600)
    sp = het_params(n, ROE, 9601)
    worst = []
    for bc in (PER, FIX):
        def F(_t, v):
            r = v.reshape(-1, 3)
            x, y, z = r[:, 0], r[:, 1], r[:, 2]
            if bc == PER:
                xl, xr = np.roll(x, 1), np.roll(x, -1)
            else:
                xl, xr = np.concatenate(([0.0], x[:-1])), np.concatenate((x[1:], [0.0]))
            out = np.empty_like(r)
            out[:, 0] = -y - z + sp[:, 3] * (xl - 2 * x + xr)
            out[:, 1] = x + sp[:, 0] * y
            out[:, 2] = sp[:, 1] + z * (x - sp[:, 2])
            return out.reshape(-1)
        ref = solve_ivp(F, (0, T), y0.reshape(-1), method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1].reshape(-1, 3)
        errs = [cf.rel_inf(oracle.rk4_integrate_het(y0, sp, ROE, bc, dt, int(round(T / dt)), lib=lib), ref)
                for dt in (0.025, 0.0125)]
        worst.append(float(np.log2(errs[0] / errs[1])))
    ok = all(3.8 < p < 4.3 for p in worst)
    return ok, f"heterogeneous Roessler observed orders {worst}"


def pin_het_uniform_equals_homogeneous(lib, n=33, nsteps=100):
    y0 = ci.uniform_state(n, 3, seed=9700)
    sp = np.tile([0.2, 1.0, 9.0, 1.3], (n, 1))
    a = oracle.rk4_integrate_het(y0, sp, ROE, FIX, 0.01, nsteps, lib=lib)
    b = oracle.rk4_integrate(y0, ROE, FIX, 0.01, nsteps, oracle.params(kappa=1.3), lib=lib)
    err = cf.rel_inf(a, b)
    return err < 1e-13, f"uniform heterogeneous vs homogeneous rel err {err:.2e}"


ALL_PINS = [
    ("harmonic_modal_per", lambda lib: pin_harmonic_modal(lib, bc=PER)),
    ("harmonic_modal_fix", lambda lib: pin_harmonic_modal(lib, bc=FIX)),
    ("harmonic_order4_per", lambda lib: pin_harmonic_order4(lib, bc=PER)),
    ("harmonic_order4_fix", lambda lib: pin_harmonic_order4(lib, bc=FIX)),
    ("harmonic_energy_per", lambda lib: pin_harmonic_energy(lib, bc=PER)),
    ("harmonic_energy_fix", lambda lib: pin_harmonic_energy(lib, bc=FIX)),
    ("roessler_fixed_point", pin_roessler_fixed_point),
    ("roessler_dop853_per", lambda lib: pin_roessler_vs_dop853(lib, bc=PER)),
    ("roessler_dop853_fix", lambda lib: pin_roessler_vs_dop853(lib, bc=FIX, kappa=1.7)),
    ("roessler_uniform", pin_roessler_uniform_single),
    ("roessler_decoupled", pin_roessler_decoupled),
    ("brute_roe_per", lambda lib: pin_brute_force(lib, model=ROE, bc=PER)),
    ("brute_roe_fix", lambda lib: pin_brute_force(lib, model=ROE, bc=FIX)),
    ("brute_har_fix", lambda lib: pin_brute_force(lib, model=HAR, bc=FIX)),
    ("shift", pin_shift_invariance),
    ("reflection", pin_reflection),
    ("cone", pin_dependency_cone),
    ("tableau_orders", pin_tableau_orders),
    ("nnn_modal", pin_nnn_modal),
    ("nnn_energy_fixed", pin_nnn_energy_fixed),
    ("nnn_cone", pin_nnn_cone),
    ("dopri5_nnn_cone", pin_dopri5_nnn_cone),
    ("nnn_dop853_fix", lambda lib: pin_roessler_vs_dop853(lib, bc=FIX, kappa=1.2, kappa2=0.7)),
    ("nnn_brute_per", lambda lib: pin_brute_force(lib, n=5, model=ROE, bc=PER, kappa2=0.9)),
    ("nnn_brute_fix", lambda lib: pin_brute_force(lib, n=6, model=HAR, bc=FIX, kappa2=0.9)),
    ("het_decoupled", pin_het_decoupled),
    ("het_harmonic_eigen", pin_het_harmonic_eigen),
    ("het_roessler_dop853", pin_het_roessler_dop853),
    ("het_uniform", pin_het_uniform_equals_homogeneous),
]
