"""Deterministic and classical radiation-reaction models of Sec. 2.4 (oracle, test-only).

Eq. (Losses_classical): d gamma_d/dt = -P[eta_d]/(m c^2), P = P_c g(eta), with
P_c = (4 pi m c^3/(3 lambda_c)) alpha eta^2 = (2/3) alpha eta^2 m c^2 omega_C (lambda_c = h/(m c)).
For an ultra-relativistic particle perpendicular to a uniform cB, eta = gamma cB/E_s
(Sec. 2.1), so in units of hbar/(m c^2):  d gamma/dt = -(2/3) alpha (gamma cB)^2 g(gamma cB).
The classical model sets g = 1 (Sec. 4), with the closed form
gamma_c(t) = gamma0 / (1 + (2/3) alpha cB^2 gamma0 t).
"""
from __future__ import annotations

import numpy as np

from . import ALPHA, g as g_quadrature


def gamma_classical(gamma0: float, cB: float, t):
    return gamma0 / (1.0 + (2.0 / 3.0) * ALPHA * cB * cB * gamma0 * np.asarray(t, dtype=np.float64))


def power(eta: float, g=g_quadrature) -> float:
    """Radiated power P(eta) = (2/3) alpha eta^2 g(eta), units m c^2 omega_C (Sec. 2.1)."""
    return (2.0 / 3.0) * ALPHA * eta * eta * g(eta)


def gamma_deterministic(gamma0: float, cB: float, t_end: float, n: int = 400, g=g_quadrature):
    """Classical RK4 integration of Eq. (Losses_classical); returns (t, gamma) on n+1 points."""
    t = np.linspace(0.0, t_end, n + 1)
    h = t[1] - t[0]
    y = np.empty(n + 1)
    y[0] = gamma0

    def rhs(gam):
        return -power(gam * cB, g)

    for i in range(n):
        k1 = rhs(y[i])
        k2 = rhs(y[i] + 0.5 * h * k1)
        k3 = rhs(y[i] + 0.5 * h * k2)
        k4 = rhs(y[i] + h * k3)
        y[i + 1] = y[i] + h * (k1 + 2 * k2 + 2 * k3 + k4) / 6.0
    return t, y
