"""The CPU oracle against what the paper and the mathematics fix (no GPU needed).

Every pin in ``oracle_pins.ALL_PINS`` must hold for the oracle as committed.  The mutation
test then plants one plausible mistake at a time in a copy of the oracle's C source (a
dropped term, a wrong sign, a wrong index, a wrong tableau entry, a wrong boundary, a wrong
energy bond), rebuilds it, and requires that at least one pin fails for every mutant.
"""
import numpy as np
import pytest

import chain_inputs as ci
import oracle
import oracle_pins as P


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("name,pin", P.ALL_PINS, ids=[n for n, _ in P.ALL_PINS])
def test_pin(lib, name, pin):
    ok, detail = pin(lib)
    assert ok, detail


def test_half_norm2_is_unit_harmonic_energy(lib):
    """For D=2, (1/2) sum |r|^2 is the harmonic energy with kappa = 0, omega0 = 1, which the
    modal energy pin fixes independently."""
    y = ci.uniform_state(37, 2, seed=11)
    e = oracle.energy_harmonic(y, oracle.PERIODIC, oracle.params(kappa=0.0, omega0=1.0), lib=lib)
    assert oracle.half_norm2(y, lib=lib) == pytest.approx(e, rel=1e-15)


def test_tiny_chains(lib):
    """N = 1 and 2 periodic use wrapped self- and neighbour indices; the harmonic chain's
    modal form covers them."""
    for n in (1, 2, 3):
        ok, detail = P.pin_harmonic_modal(lib, n=n, nsteps=200)
        assert ok, detail
        ok, detail = P.pin_harmonic_modal(lib, n=n, bc=oracle.FIXED, nsteps=200)
        assert ok, detail


def test_zero_steps_identity(lib):
    y0 = ci.uniform_state(10, 3)
    assert np.array_equal(oracle.rk4_integrate(y0, nsteps=0, lib=lib), y0)


def test_batch_equals_separate_chains(lib):
    lengths = np.array([5, 9, 1, 16])
    kap = np.array([0.5, 1.0, 2.0, 1.5])
    bcs = np.array([0, 1, 0, 1])
    y0 = ci.uniform_state(int(lengths.sum()), 3, seed=99)
    got = oracle.batch_rk4_integrate(y0, lengths, kap, bcs, nsteps=20, lib=lib)
    off = 0
    for n, k, b in zip(lengths, kap, bcs):
        one = oracle.rk4_integrate(y0[off:off + n], oracle.ROESSLER, int(b), 0.01, 20,
                                   oracle.params(kappa=float(k)), lib=lib)
        assert np.array_equal(one, got[off:off + n])
        off += n


# (label, original text, planted mistake) -- each original must occur exactly once
MUTANTS = [
    ("drop coupling", "ki[0] = -y - z + p->kappa * lap + p->kappa2 * lap2;", "ki[0] = -y - z + p->kappa2 * lap2;"),
    ("drop second-neighbour coupling", "ki[0] = -y - z + p->kappa * lap + p->kappa2 * lap2;",
     "ki[0] = -y - z + p->kappa * lap;"),
    ("second-neighbour index", "int64_t ir = (i + 2) % n;", "int64_t ir = (i + 1) % n;"),
    ("second-neighbour fixed ghost", "*xl = (i - 2 < 0) ? 0.0 : r[(i - 2) * D];", "*xl = (i - 2 < 0) ? r[0] : r[(i - 2) * D];"),
    ("harmonic second-neighbour sign", "q + p->kappa * lap + p->kappa2 * lap2;", "q + p->kappa * lap - p->kappa2 * lap2;"),
    ("energy second-neighbour ghost bonds", "const int64_t first = (bc == ORC_PERIODIC) ? 0 : -2;",
     "const int64_t first = 0;"),
    ("sign f_y", "ki[1] = x + p->a * y;", "ki[1] = x - p->a * y;"),
    ("transposed f_z", "ki[2] = p->b + z * (x - p->c);", "ki[2] = p->b + x * (z - p->c);"),
    ("laplacian index", "double lap = xl - 2.0 * x + xr;   /* Eq. (7)", "double lap = xl - 2.0 * x + xl;   /* Eq. (7)"),
    ("heterogeneous laplacian index", "double lap = xl - 2.0 * x + xr;\n      ki[0] = -y - z + q[3]",
     "double lap = xl - 2.0 * x + xl;\n      ki[0] = -y - z + q[3]"),
    ("harmonic omega not squared", "ki[1] = -p->omega0 * p->omega0 * q", "ki[1] = -p->omega0 * q"),
    ("harmonic coupling sign", "q + p->kappa * lap + p->kappa2 * lap2;", "q - p->kappa * lap + p->kappa2 * lap2;"),
    ("periodic wrap", "int64_t il = (i == 0) ? n - 1 : i - 1;", "int64_t il = (i == 0) ? 0 : i - 1;"),
    ("free end instead of fixed", "*xl = (i == 0) ? 0.0 : r[(i - 1) * D];", "*xl = (i == 0) ? r[0] : r[(i - 1) * D];"),
    ("weights b", "RK4_B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0}",
     "RK4_B[4] = {1.0 / 6.0, 1.0 / 6.0, 1.0 / 2.0, 1.0 / 6.0}"),
    ("heterogeneous weights b", "double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0}",
     "double b[4] = {1.0 / 6.0, 1.0 / 6.0, 1.0 / 2.0, 1.0 / 6.0}"),
    ("heterogeneous stage coefficient", "double a[4] = {0.0, 0.5, 0.5, 1.0};", "double a[4] = {0.0, 0.5, 1.0, 1.0};"),
    ("a43", "0.0, 0.0, 1.0, 0.0};", "0.0, 0.0, 0.5, 0.0};"),
    ("stage sum truncated", "for (int m = 0; m < j; ++m) sum +=", "for (int m = (j > 0 ? j - 1 : 0); m < j; ++m) sum +="),
    ("stage dt dropped", "sum += A[j * s + m] * dt * k", "sum += A[j * s + m] * k"),
    ("combine from stage state", "m < s; ++m) sum += b[m] * dt * k[(int64_t)m * len + e];\n      y[e] = y[e] + sum;",
     "m < s; ++m) sum += b[m] * dt * k[(int64_t)m * len + e];\n      y[e] = r[e] + sum;"),
    ("heterogeneous combine from stage state",
     "m < 4; ++m) sum += b[m] * dt * k[(int64_t)m * len + e];\n      y[e] = y[e] + sum;",
     "m < 4; ++m) sum += b[m] * dt * k[(int64_t)m * len + e];\n      y[e] = r[e] + sum;"),
    ("stale neighbours", "rhs(model, bc, n, &p, r, k + (int64_t)j * len);",
     "rhs(model, bc, n, &p, (j == s - 1) ? y : r, k + (int64_t)j * len);"),
    ("energy ghost bonds", "for (int64_t i = -1; i < n; ++i) {", "for (int64_t i = 0; i < n - 1; ++i) {"),
    ("energy periodic bond", "y[2 * ((i + 1) % n)] - y[2 * i]", "y[2 * ((i + 2) % n)] - y[2 * i]"),
    ("energy potential", "0.5 * w2 * q * q", "0.5 * q * q"),
    ("heterogeneous a/b swapped", "ki[1] = x + q[0] * y;", "ki[1] = x + q[1] * y;"),
    ("heterogeneous neighbour's parameters", "const double *q = sp + 4 * i;", "const double *q = sp + 4 * ((i + 1) % n);"),
    ("heterogeneous coupling dropped", "ki[0] = -y - z + q[3] * lap;", "ki[0] = -y - z + lap;"),
    ("heterogeneous harmonic omega", "ki[1] = -q[0] * ri[0] + q[1] * lap;", "ki[1] = -q[1] * ri[0] + q[1] * lap;"),
]


@pytest.mark.parametrize("label,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, label, orig, bad):
    src = open(oracle._SRC).read()
    assert src.count(orig) == 1, f"mutation anchor for '{label}' not unique"
    msrc = tmp_path / "mutant.c"
    msrc.write_text(src.replace(orig, bad))
    so = oracle.build(force=True, src=str(msrc), out=str(tmp_path / "libmutant.so"))
    mlib = oracle.load(so)
    failed = []
    for name, pin in P.ALL_PINS:
        try:
            ok, _ = pin(mlib)
        except Exception:  # a mutant that crashes a pin is caught too
            ok = False
        if not ok:
            failed.append(name)
    if not failed:
        # the half-norm / energy cross-check is the remaining pin
        y = ci.uniform_state(37, 2, seed=11)
        e = oracle.energy_harmonic(y, 0, oracle.params(kappa=0.0, omega0=1.0), lib=mlib)
        if abs(oracle.half_norm2(y, lib=mlib) - e) > 1e-14 * abs(e):
            failed.append("half_norm2")
    assert failed, f"mutant '{label}' passed every pin"
