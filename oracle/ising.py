"""Closed forms of the square-lattice Ising model (J = 1, H = -sum s_i s_j).

TEST INFRASTRUCTURE ONLY: these are the pins of the CTMRG oracle, not part of
the method. Each quantity is given in two independent forms so that a typo in
one is caught by the other.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, special

BETA_C = 0.5 * np.log(1.0 + np.sqrt(2.0))


def onsager_lnz(beta):
    """-beta f per site, Onsager's single-integral form:
    ln(2 cosh 2b) + (1/pi) int_0^{pi/2} ln[(1 + sqrt(1 - k^2 sin^2 t)) / 2] dt,
    k = 2 sinh 2b / cosh^2 2b."""
    k = 2.0 * np.sinh(2 * beta) / np.cosh(2 * beta) ** 2
    val, _ = integrate.quad(
        lambda t: np.log(0.5 * (1.0 + np.sqrt(1.0 - (k * np.sin(t)) ** 2))),
        0.0, 0.5 * np.pi, epsabs=1e-14, epsrel=1e-14, limit=200)
    return np.log(2.0 * np.cosh(2 * beta)) + val / np.pi


def onsager_lnz_double(beta, n=512):
    """-beta f per site, double-integral form:
    ln 2 + 1/(8 pi^2) int int ln[cosh^2 2b - sinh 2b (cos t1 + cos t2)],
    evaluated with an n x n periodic trapezoid rule (spectrally accurate for
    the analytic periodic integrand away from the critical point)."""
    t = 2.0 * np.pi * np.arange(n) / n
    c = np.cos(t)
    arg = np.cosh(2 * beta) ** 2 - np.sinh(2 * beta) * (c[:, None] + c[None, :])
    return np.log(2.0) + 0.5 * np.mean(np.log(arg))


def yang_m(beta):
    """Spontaneous magnetisation (1 - sinh^-4 2b)^(1/8) for b > b_c, else 0."""
    if beta <= BETA_C:
        return 0.0
    return (1.0 - np.sinh(2 * beta) ** -4) ** 0.125


def nn_correlation(beta):
    """<s_i s_j> for nearest neighbours = (1/2) d(-beta f)/d beta, closed form
    (1/2) coth 2b [1 + (2/pi)(2 tanh^2 2b - 1) K(k)], K the complete elliptic
    integral of the first kind with modulus k = 2 sinh 2b / cosh^2 2b."""
    k = 2.0 * np.sinh(2 * beta) / np.cosh(2 * beta) ** 2
    K = special.ellipk(k * k)
    return 0.5 / np.tanh(2 * beta) * (
        1.0 + 2.0 / np.pi * (2.0 * np.tanh(2 * beta) ** 2 - 1.0) * K)
