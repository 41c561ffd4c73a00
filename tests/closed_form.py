"""Closed-form solutions of the linear harmonic chain, used to pin the oracle and the GPU path.

The harmonic chain q_i' = p_i, p_i' = -omega0^2 q_i + kappa (q_{i-1} - 2 q_i + q_{i+1}) belongs
to the paper's class Eq. (2) (oscillator chains, Sec. 2.1).  Its coupling matrix is
diagonalised by known normal modes, so nothing here evaluates the chain's slope field:

* periodic ends: Fourier modes exp(2 pi i m j / N), omega_m^2 = omega0^2 + 4 kappa sin^2(pi m / N);
* fixed ends (q_0 = q_{N+1} = 0): sine modes sin(pi m j / (N+1)), m = 1..N,
  omega_m^2 = omega0^2 + 4 kappa sin^2(pi m / (2 (N+1))).

In a mode, (q, p)' = A (q, p) with A = [[0, 1], [-w^2, 0]] and A^2 = -w^2 I, so the classical
RK4 polynomial P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 at z = dt A collapses to
R = alpha I + beta dt A with h = w dt, alpha = 1 - h^2/2 + h^4/24, beta = 1 - h^2/6.  In scaled
coordinates (q, p / w) R is sqrt(rho) times a rotation by theta = atan2(beta h, alpha), with
rho = alpha^2 + beta^2 h^2 = 1 - h^6/72 + h^8/576, so n steps are rho^(n/2) Rot(n theta), and
each mode's energy is multiplied by exactly rho^n.  The exact flow is the rotation by w t.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def mode_frequencies(n: int, bc: int, kappa: float, omega0: float, kappa2: float = 0.0) -> np.ndarray:
    """omega_m for the modes in the order the transform below produces them.  Second-neighbour
    coupling kappa2 keeps the Fourier modes (periodic ends only): it adds
    4 kappa2 sin^2(2 pi m / N)."""
    if bc == 0:
        m = np.arange(n)
        return np.sqrt(omega0 ** 2 + 4.0 * kappa * np.sin(np.pi * m / n) ** 2
                       + 4.0 * kappa2 * np.sin(2.0 * np.pi * m / n) ** 2)
    if kappa2 != 0.0:
        raise ValueError("second-neighbour coupling with fixed ends has no sine-mode closed form")
    m = np.arange(1, n + 1)
    return np.sqrt(omega0 ** 2 + 4.0 * kappa * np.sin(np.pi * m / (2.0 * (n + 1))) ** 2)


def _forward(v: np.ndarray, bc: int):
    return sfft.fft(v) if bc == 0 else sfft.dst(v, type=1)


def _inverse(v, bc: int) -> np.ndarray:
    return np.real(sfft.ifft(v)) if bc == 0 else sfft.idst(v, type=1)


def _evolve(y0: np.ndarray, bc: int, kappa: float, omega0: float, amp: np.ndarray, ang: np.ndarray,
            kappa2: float = 0.0) -> np.ndarray:
    """Apply amp * Rot(ang) in scaled mode coordinates (q, p / w) to every mode."""
    y0 = np.asarray(y0, dtype=np.float64).reshape(-1, 2)
    n = y0.shape[0]
    w = mode_frequencies(n, bc, kappa, omega0, kappa2)
    qh = _forward(y0[:, 0], bc)
    sh = _forward(y0[:, 1], bc) / w
    c, s = np.cos(ang), np.sin(ang)
    q1 = amp * (c * qh + s * sh)
    s1 = amp * (-s * qh + c * sh)
    out = np.empty_like(y0)
    out[:, 0] = _inverse(q1, bc)
    out[:, 1] = _inverse(s1 * w, bc)
    return out


def rk4_modal(y0, bc: int, kappa: float, omega0: float, dt: float, nsteps: int, kappa2: float = 0.0) -> np.ndarray:
    """Exact (up to rounding) result of nsteps classical RK4 steps on the harmonic chain."""
    n = np.asarray(y0).reshape(-1, 2).shape[0]
    w = mode_frequencies(n, bc, kappa, omega0, kappa2)
    h = w * dt
    alpha = 1.0 - h ** 2 / 2.0 + h ** 4 / 24.0
    beta = 1.0 - h ** 2 / 6.0
    rho = alpha ** 2 + (beta * h) ** 2
    theta = np.arctan2(beta * h, alpha)
    return _evolve(y0, bc, kappa, omega0, rho ** (nsteps / 2.0), nsteps * theta, kappa2)


def exact_flow(y0, bc: int, kappa: float, omega0: float, t: float) -> np.ndarray:
    """The continuous solution at time t (each mode rotates by omega_m t)."""
    n = np.asarray(y0).reshape(-1, 2).shape[0]
    w = mode_frequencies(n, bc, kappa, omega0)
    return _evolve(y0, bc, kappa, omega0, np.ones_like(w), w * t)


def modal_energy(y0, bc: int, kappa: float, omega0: float, kappa2: float = 0.0) -> np.ndarray:
    """Per-mode energies (1/2)(|p_m|^2 + w_m^2 |q_m|^2), normalised so they sum to H."""
    y0 = np.asarray(y0, dtype=np.float64).reshape(-1, 2)
    n = y0.shape[0]
    w = mode_frequencies(n, bc, kappa, omega0, kappa2)
    qh = _forward(y0[:, 0], bc)
    ph = _forward(y0[:, 1], bc)
    # Parseval factors: sum |v|^2 = (1/N) sum |fft v|^2;  for DST-I: sum |v|^2 = sum |dst v|^2 / (2 (N+1))
    norm = 1.0 / n if bc == 0 else 1.0 / (2.0 * (n + 1))
    return 0.5 * norm * (np.abs(ph) ** 2 + (w ** 2) * np.abs(qh) ** 2)


def rk4_energy(y0, bc: int, kappa: float, omega0: float, dt: float, nsteps: int) -> float:
    """Energy after nsteps RK4 steps: sum_m E_m(0) rho(h_m)^n, exact up to rounding."""
    n = np.asarray(y0).reshape(-1, 2).shape[0]
    w = mode_frequencies(n, bc, kappa, omega0)
    h = w * dt
    rho = 1.0 - h ** 6 / 72.0 + h ** 8 / 576.0
    return float(np.sum(modal_energy(y0, bc, kappa, omega0) * rho ** nsteps))


def rel_inf(a, b) -> float:
    """max |a - b| / max |b| (the infinity-norm relative error used throughout)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))
