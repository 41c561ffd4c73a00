/*
 * rk4_oracle.c -- serial FP64 CPU oracle for explicit Runge-Kutta integration of a
 * one-dimensional chain with nearest-neighbour coupling (Mulansky, "Optimizing
 * Large-Scale ODE Simulations", arXiv:1412.0544).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg may load this file.  It shares no code, header or constant with the
 * CUDA library, and the library never calls it.
 *
 * What it computes, by the paper's own definitions, with no blocking or fusion:
 *   - the homogeneous nearest-neighbour ODE of Eq. (2), r_i' = f(r_i) + g(r_i, r_{i-1}, r_{i+1});
 *   - f, g of the coupled Roessler chain, Eqs. (6)-(7), with a coupling strength kappa
 *     multiplying g (kappa = 1 is the paper's chain), optionally plus a next-nearest-neighbour
 *     term kappa2 (x_{i-2} - 2 x_i + x_{i+2}) (the longer coupling range of Sec. 5; kappa2 = 0
 *     is the paper's chain);
 *   - a harmonic (linear oscillator) chain from the same class (the oscillator chains of
 *     Sec. 2.1), with q' = p, p' = -omega0^2 q + kappa (q_{i-1} - 2 q_i + q_{i+1})
 *     (+ kappa2 (q_{i-2} - 2 q_i + q_{i+2}));
 *   - periodic ends r_0 = r_N, r_{N+1} = r_1 (Sec. 3.1), or fixed ends r_0 = r_{N+1} = 0
 *     (not in the paper: a Dirichlet reading);
 *   - an explicit Runge-Kutta step in the paper's order, Eqs. (3)-(5): for each stage j the
 *     stage state r' = r + sum_{m<j} a_{j,m} dt k^m, then k^j = F(r'); finally
 *     r <- r + sum_m b_m dt k^m.  Each of these is one full sweep over the chain, which is
 *     the paper's "standard implementation" (2s sweeps per step, Sec. 2.2);
 *   - the classical fourth-order tableau (Sec. 2, which cites Press et al. for it):
 *     c = (0, 1/2, 1/2, 1), a21 = a32 = 1/2, a43 = 1, b = (1/6, 1/3, 1/3, 1/6);
 *   - the harmonic chain's energy and the half squared norm (1/2) sum |r_i|^2;
 *   - heterogeneous chains, Eq. (1): site-dependent f_i and g_i through per-site parameters
 *     (Roessler: a_i, b_i, c_i, kappa_i; harmonic: omega_i^2, kappa_i), with
 *     g_i = kappa_i (x_{i-1} - 2 x_i + x_{i+1}).
 * The system is autonomous, so stage times c_j dt are carried but unused (the garbled
 * time arguments of Eq. (3) are read as t + c_j dt for both f and g).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math, no FMA contraction).
 * Parity pins: see the oracle tests (closed-form harmonic modes, order-4 convergence,
 * energy, brute force, Roessler fixed point, invariants, dependency cone).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_ROESSLER = 0, ORC_HARMONIC = 1 };
enum { ORC_PERIODIC = 0, ORC_FIXED = 1 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

#define ORC_MAX_STAGES 16

/* parameter vector layout shared with the Python wrapper: a, b, c, kappa, omega0, kappa2 */
typedef struct {
  double a, b, c, kappa, omega0, kappa2;
} orc_params;

int oracle_dim(int model) {
  if (model == ORC_ROESSLER) return 3;
  if (model == ORC_HARMONIC) return 2;
  return 0;
}

/* Coupling coordinate (x for Roessler, q for the harmonic chain) of the left and right
 * neighbours of site i, resolved by the boundary condition. */
static void neighbours(int bc, int64_t n, int D, const double *r, int64_t i, double *xl, double *xr) {
  if (bc == ORC_PERIODIC) {
    int64_t il = (i == 0) ? n - 1 : i - 1;
    int64_t ir = (i == n - 1) ? 0 : i + 1;
    *xl = r[il * D];
    *xr = r[ir * D];
  } else {
    *xl = (i == 0) ? 0.0 : r[(i - 1) * D];
    *xr = (i == n - 1) ? 0.0 : r[(i + 1) * D];
  }
}

/* Coupling coordinate of the second neighbours i-2 and i+2 (zero beyond fixed ends). */
static void neighbours2(int bc, int64_t n, int D, const double *r, int64_t i, double *xl, double *xr) {
  if (bc == ORC_PERIODIC) {
    int64_t il = ((i - 2) % n + n) % n;
    int64_t ir = (i + 2) % n;
    *xl = r[il * D];
    *xr = r[ir * D];
  } else {
    *xl = (i - 2 < 0) ? 0.0 : r[(i - 2) * D];
    *xr = (i + 2 > n - 1) ? 0.0 : r[(i + 2) * D];
  }
}

/* Eq. (3): k_i = f(r_i) + g(r_i, r_{i-1}, r_{i+1}) for every site, one sweep. */
static void rhs(int model, int bc, int64_t n, const orc_params *p, const double *r, double *k) {
  const int D = oracle_dim(model);
  for (int64_t i = 0; i < n; ++i) {
    double xl, xr, xl2, xr2;
    neighbours(bc, n, D, r, i, &xl, &xr);
    neighbours2(bc, n, D, r, i, &xl2, &xr2);
    const double *ri = r + i * D;
    double *ki = k + i * D;
    if (model == ORC_ROESSLER) {
      double x = ri[0], y = ri[1], z = ri[2];
      double lap = xl - 2.0 * x + xr;   /* Eq. (7), first component */
      double lap2 = xl2 - 2.0 * x + xr2; /* second neighbours */
      ki[0] = -y - z + p->kappa * lap + p->kappa2 * lap2; /* Eq. (6) f_x plus coupling */
      ki[1] = x + p->a * y;                               /* Eq. (6) f_y */
      ki[2] = p->b + z * (x - p->c);                      /* Eq. (6) f_z */
    } else {
      double q = ri[0], pm = ri[1];
      double lap = xl - 2.0 * q + xr;
      double lap2 = xl2 - 2.0 * q + xr2;
      ki[0] = pm;
      ki[1] = -p->omega0 * p->omega0 * q + p->kappa * lap + p->kappa2 * lap2;
    }
  }
}

/* Eq. (1): the heterogeneous slope field; sp holds P parameters per site (P = 4 Roessler:
 * a, b, c, kappa; P = 2 harmonic: omega^2, kappa). */
static void rhs_het(int model, int bc, int64_t n, const double *sp, const double *r, double *k) {
  const int D = oracle_dim(model);
  for (int64_t i = 0; i < n; ++i) {
    double xl, xr;
    neighbours(bc, n, D, r, i, &xl, &xr);
    const double *ri = r + i * D;
    double *ki = k + i * D;
    if (model == ORC_ROESSLER) {
      const double *q = sp + 4 * i;
      double x = ri[0], y = ri[1], z = ri[2];
      double lap = xl - 2.0 * x + xr;
      ki[0] = -y - z + q[3] * lap;
      ki[1] = x + q[0] * y;
      ki[2] = q[1] + z * (x - q[2]);
    } else {
      const double *q = sp + 2 * i;
      double lap = xl - 2.0 * ri[0] + xr;
      ki[0] = ri[1];
      ki[1] = -q[0] * ri[0] + q[1] * lap;
    }
  }
}

/* Classical RK4 (Eqs. (3)-(5)) on a heterogeneous chain, full sweeps. */
int oracle_rk4_integrate_het(int model, int bc, int64_t n, const double *sp, double dt, int64_t nsteps, double *y) {
  static const double a[4] = {0.0, 0.5, 0.5, 1.0}; /* a_{j,j-1}; the other entries are zero */
  static const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const int D = oracle_dim(model);
  if (D == 0 || n < 1 || (bc != ORC_PERIODIC && bc != ORC_FIXED)) return ORC_EINVAL;
  const int64_t len = n * D;
  double *k = (double *)malloc(sizeof(double) * (size_t)len * 4);
  double *r = (double *)malloc(sizeof(double) * (size_t)len);
  if (!k || !r) {
    free(k);
    free(r);
    return ORC_ENOMEM;
  }
  for (int64_t step = 0; step < nsteps; ++step) {
    for (int j = 0; j < 4; ++j) {
      for (int64_t e = 0; e < len; ++e) r[e] = y[e] + (j > 0 ? a[j] * dt * k[(int64_t)(j - 1) * len + e] : 0.0);
      rhs_het(model, bc, n, sp, r, k + (int64_t)j * len);
    }
    for (int64_t e = 0; e < len; ++e) {
      double sum = 0.0;
      for (int m = 0; m < 4; ++m) sum += b[m] * dt * k[(int64_t)m * len + e];
      y[e] = y[e] + sum;
    }
  }
  free(k);
  free(r);
  return ORC_OK;
}

/* One chain, any explicit tableau with s stages: A is s x s row-major (strictly lower
 * part used), b has s weights.  y holds n*D values (site-major, components contiguous,
 * the paper's Fig. 1 layout) and is advanced nsteps steps in place. */
int oracle_rk_integrate(int model, int bc, int64_t n, const double *prm, int s, const double *A,
                        const double *b, double dt, int64_t nsteps, double *y) {
  const int D = oracle_dim(model);
  if (D == 0 || n < 1 || s < 1 || s > ORC_MAX_STAGES || (bc != ORC_PERIODIC && bc != ORC_FIXED))
    return ORC_EINVAL;
  orc_params p = {prm[0], prm[1], prm[2], prm[3], prm[4], prm[5]};
  const int64_t len = n * D;
  double *k = (double *)malloc(sizeof(double) * (size_t)len * (size_t)s);
  double *r = (double *)malloc(sizeof(double) * (size_t)len);
  if (!k || !r) {
    free(k);
    free(r);
    return ORC_ENOMEM;
  }
  for (int64_t step = 0; step < nsteps; ++step) {
    for (int j = 0; j < s; ++j) {
      /* Eq. (4): stage state from the step's start and the earlier stage slopes */
      for (int64_t e = 0; e < len; ++e) {
        double sum = 0.0;
        for (int m = 0; m < j; ++m) sum += A[j * s + m] * dt * k[(int64_t)m * len + e];
        r[e] = y[e] + sum;
      }
      /* Eq. (3): slope of stage j */
      rhs(model, bc, n, &p, r, k + (int64_t)j * len);
    }
    /* Eq. (5): combine the stage slopes */
    for (int64_t e = 0; e < len; ++e) {
      double sum = 0.0;
      for (int m = 0; m < s; ++m) sum += b[m] * dt * k[(int64_t)m * len + e];
      y[e] = y[e] + sum;
    }
  }
  free(k);
  free(r);
  return ORC_OK;
}

/* Classical fourth-order Runge-Kutta tableau. */
static const double RK4_A[16] = {0.0, 0.0, 0.0, 0.0, 0.5, 0.0, 0.0, 0.0,
                                 0.0, 0.5, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0};
static const double RK4_B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

int oracle_rk4_integrate(int model, int bc, int64_t n, const double *prm, double dt, int64_t nsteps,
                         double *y) {
  return oracle_rk_integrate(model, bc, n, prm, 4, RK4_A, RK4_B, dt, nsteps, y);
}

/* The slope field F(r) alone (one Eq. (3) sweep), exposed for tests. */
int oracle_rhs(int model, int bc, int64_t n, const double *prm, const double *r, double *k) {
  if (oracle_dim(model) == 0 || n < 1) return ORC_EINVAL;
  orc_params p = {prm[0], prm[1], prm[2], prm[3], prm[4], prm[5]};
  rhs(model, bc, n, &p, r, k);
  return ORC_OK;
}

/* Harmonic-chain energy H = sum_i (p_i^2/2 + omega0^2 q_i^2/2) + kappa/2 sum_bonds (dq)^2
 * + kappa2/2 sum_second-bonds (q_{i+2} - q_i)^2.  Periodic: N bonds of each kind (indices mod
 * N).  Fixed: every bond with at least one end in the chain, the other end possibly a zero
 * ghost (N+1 nearest bonds, N+2 second-neighbour bonds).  H is the Hamiltonian whose
 * equations of motion are the harmonic chain above. */
static double q_at(int bc, int64_t n, const double *y, int64_t i) {
  if (bc == ORC_PERIODIC) return y[2 * (((i % n) + n) % n)];
  return (i < 0 || i >= n) ? 0.0 : y[2 * i];
}

double oracle_energy_harmonic(int bc, int64_t n, const double *prm, const double *y) {
  const double kappa = prm[3], w2 = prm[4] * prm[4], kappa2 = prm[5];
  double e = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double q = y[2 * i], pm = y[2 * i + 1];
    e += 0.5 * pm * pm + 0.5 * w2 * q * q;
  }
  if (bc == ORC_PERIODIC) {
    for (int64_t i = 0; i < n; ++i) {
      double d = y[2 * ((i + 1) % n)] - y[2 * i];
      e += 0.5 * kappa * d * d;
    }
  } else {
    for (int64_t i = -1; i < n; ++i) {
      double ql = (i < 0) ? 0.0 : y[2 * i];
      double qr = (i + 1 >= n) ? 0.0 : y[2 * (i + 1)];
      double d = qr - ql;
      e += 0.5 * kappa * d * d;
    }
  }
  if (kappa2 != 0.0) {
    const int64_t first = (bc == ORC_PERIODIC) ? 0 : -2;
    for (int64_t i = first; i < n; ++i) {
      double d = q_at(bc, n, y, i + 2) - q_at(bc, n, y, i);
      e += 0.5 * kappa2 * d * d;
    }
  }
  return e;
}

/* (1/2) sum_i |r_i|^2 over all components: a monitored norm for the dissipative
 * Roessler chain (not a conserved quantity). */
double oracle_half_norm2(int64_t len, const double *y) {
  double e = 0.0;
  for (int64_t j = 0; j < len; ++j) e += y[j] * y[j];
  return 0.5 * e;
}
