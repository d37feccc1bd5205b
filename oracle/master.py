"""Direct numerical solution of the master equations of Sec. 2.4 (Eqs. master_electrons and
master_photons) for electrons moving perpendicular to a uniform magnetic field, photon emission
only (pair creation neglected, as for the mean-loss identity Eq. Losses_QED).

TEST INFRASTRUCTURE, part of the oracle: only the tests import it.  The Monte-Carlo step is
checked against it (Sec. 4 compares the Monte-Carlo spectra with such a direct solution).

Physics (Sec. 2.4): an electron of Lorentz factor gamma perpendicular to cB has eta = gamma cB
(ultra-relativistic, the regime the master equations hold in) and emits a photon of energy eps,
chi = eps cB / 2, at the rate density

    w(gamma, eps) = (sqrt3 alpha / 2 pi) (eta / gamma) F(eta, chi) / chi * (cB / 2)

(time in hbar/(m c^2)), whose integral over eps < gamma is lambda_gamma = (sqrt3 alpha/2pi)
(eta/gamma) h(eta) of Eq. rate_photons.  Eq. master_electrons without its pair term moves an
electron from gamma' to gamma = gamma' - eps at that rate; Eq. master_photons collects the
photons.

Scheme (Sec. 4's footnote: first-order upwinding, a time step below 0.1 Delta t_QED): gamma on
cells of width dg centred on gamma0, gamma0 - dg, ...; a photon harder than dg/2 moves the
electron's probability from its cell j to cell j - m, m = round(eps / dg) (the jump term, the
rate of each m integrated over eps in [(m - 1/2) dg, (m + 1/2) dg]); softer photons are a
continuous energy loss at the rate of their power, advected to the next lower cell by
first-order upwinding.  The photon spectrum integrates the emission rate over given photon-energy
bins.  The semi-discrete system dPhi/dt = M Phi is linear with constant coefficients, so it is
advanced exactly (a matrix exponential, with the photon counts as extra rows of the same
system) instead of by small explicit steps, whose first-order error in time would be of the
order of lambda dt.  The rate integrals use Gauss-Legendre nodes in s = eps^(1/3), which removes
the eps^(-2/3) singularity of F/chi at soft photons.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import expm

from . import ALPHA, F

_K = math.sqrt(3.0) * ALPHA / (2.0 * math.pi)
_GL_X, _GL_W = np.polynomial.legendre.leggauss(6)


def _w(gamma, eps, cB):
    """Emission rate density w(gamma, eps) (see the module docstring)."""
    eta = gamma * cB
    chi = eps * cB / 2.0
    if chi <= 0.0 or chi >= eta / 2.0:
        return 0.0
    return _K * (eta / gamma) * F(eta, chi) / chi * (cB / 2.0)


def _integral(gamma, a, b, cB, moment):
    """int_a^b eps^moment w(gamma, eps) d eps over [a, b] clipped to [0, gamma)."""
    b = min(b, gamma)
    if b <= a:
        return 0.0
    s0, s1 = a ** (1.0 / 3.0), b ** (1.0 / 3.0)
    tot = 0.0
    for x, wt in zip(_GL_X, _GL_W):
        s = 0.5 * (s1 - s0) * x + 0.5 * (s1 + s0)
        eps = s ** 3
        tot += wt * _w(gamma, eps, cB) * eps ** moment * 3.0 * s * s
    return 0.5 * (s1 - s0) * tot


def solve(gamma0: float, cB: float, t_end: float, dg: float = 4.0, photon_edges=None):
    """Phi_-(gamma, t_end) per initial electron on the cells (centres, widths dg) for electrons
    that all start at gamma0, and the photons emitted per initial electron in the bins given by
    ``photon_edges`` (ascending) during [0, t_end].  Returns (centres, phi, photons)."""
    n = int(math.floor((gamma0 - dg) / dg)) + 1
    centres = gamma0 - dg * np.arange(n)[::-1]           # ascending; the top cell is gamma0
    photon_edges = np.asarray(photon_edges if photon_edges is not None else [], dtype=np.float64)
    nb = max(0, len(photon_edges) - 1)
    # A = [[M, 0], [P, 0]]: M moves electron probability, P counts the photons emitted into each bin
    A = np.zeros((n + nb, n + nb))
    for j, g in enumerate(centres):
        out = 0.0
        for m in range(1, j + 1):  # a jump of m cells: eps in [(m - 1/2) dg, (m + 1/2) dg]
            hi = (m + 0.5) * dg if m < j else g  # the last jump takes every eps up to gamma
            r = _integral(g, (m - 0.5) * dg, hi, cB, 0)
            A[j - m, j] += r
            out += r
        A[j, j] -= out
        # soft photons: continuous loss at their power, first-order upwind into the next cell
        if j > 0:
            u = _integral(g, 0.0, 0.5 * dg, cB, 1) / dg
            A[j - 1, j] += u
            A[j, j] -= u
        for b in range(nb):
            A[n + b, j] = _integral(g, photon_edges[b], photon_edges[b + 1], cB, 0)
    x0 = np.zeros(n + nb)
    x0[n - 1] = 1.0
    x = expm(A * t_end) @ x0
    return centres, x[:n], x[n:]
