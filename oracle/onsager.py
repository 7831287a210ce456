"""Onsager's exact free energy of the 2D square-lattice Ising model at h = 0.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

ln Z / N = -beta f = ln(2 cosh 2beta)
           + (1/pi) int_0^{pi/2} ln[(1 + sqrt(1 - k^2 sin^2 t)) / 2] dt,
k = 2 sinh(2beta) / cosh^2(2beta)                       (J = 1, N -> infinity)

and the equivalent double-integral form

ln Z / N = ln 2 + 1/(2 pi^2) int_0^pi int_0^pi
           ln[cosh^2(2beta) - sinh(2beta)(cos t1 + cos t2)] dt1 dt2.

Pins: the two forms agree with each other; at the critical point
beta_c = ln(1 + sqrt 2)/2 the single integral equals 2G/pi + (1/2) ln 2 with G
Catalan's constant; beta -> 0 gives ln 2.
"""
from __future__ import annotations

import math

from scipy import integrate

BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))


def ising_ln_z_per_site(beta: float) -> float:
    """Single-integral form (quadrature to ~1e-15)."""
    k = 2.0 * math.sinh(2.0 * beta) / math.cosh(2.0 * beta) ** 2

    def integrand(t):
        return math.log(0.5 * (1.0 + math.sqrt(max(0.0, 1.0 - (k * math.sin(t)) ** 2))))

    val, _ = integrate.quad(integrand, 0.0, 0.5 * math.pi, epsabs=1e-14, epsrel=1e-14, limit=400)
    return math.log(2.0 * math.cosh(2.0 * beta)) + val / math.pi


def ising_ln_z_per_site_double(beta: float) -> float:
    """Double-integral form (slower; for cross-checks away from beta_c)."""
    c2 = math.cosh(2.0 * beta) ** 2
    s = math.sinh(2.0 * beta)

    def integrand(t2, t1):
        return math.log(c2 - s * (math.cos(t1) + math.cos(t2)))

    val, _ = integrate.dblquad(integrand, 0.0, math.pi, 0.0, math.pi, epsabs=1e-13, epsrel=1e-13)
    return math.log(2.0) + val / (2.0 * math.pi ** 2)


def ising_free_energy(beta: float) -> float:
    """f = -(1/beta) ln Z / N."""
    return -ising_ln_z_per_site(beta) / beta
