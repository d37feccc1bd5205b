"""Pins of the oracle's look-up tables and inverse-CDF samplers (Sec. 3) against quadrature
done with a different integrator.  CPU only."""
import math

import numpy as np
import pytest

import oracle as o


def eta_nodes(tab):
    p = tab.params
    return np.exp(np.linspace(math.log(p.eta_min), math.log(p.eta_max), p.n_eta))


def test_table_shapes_and_invariants(orc_tables):
    a = orc_tables.a
    P, Q = a["P"], a["Q"]
    # P saturates at 1 in double once the complement drops below 1e-16; Q keeps resolving it
    assert np.all(np.diff(P, axis=1) >= 0), "P_chi rows must not decrease"
    assert np.all(np.diff(Q, axis=1) < 0), "Q rows must decrease"
    assert np.all(Q[:, -1] < 1e-20)
    assert np.max(np.abs(P + Q - 1.0)) < 1e-14
    # the cut-off removes well under 1% of the photons (by number) at every eta
    assert np.all((P[:, 0] > 1e-3) & (P[:, 0] < 1e-2))
    Pf = a["Pf"]
    assert np.all(Pf[:, 0] == 0) and np.allclose(Pf[:, -1], 1.0)
    assert np.all(np.diff(Pf, axis=1) >= 0)


@pytest.mark.parametrize("row", [0, 60, 128, 200, 255])
def test_h_table_against_direct_quadrature(orc_tables, row):
    eta = eta_nodes(orc_tables)[row]
    assert math.exp(orc_tables.a["ln_h"][row]) == pytest.approx(o.h(eta), rel=1e-14)
    assert orc_tables.a["g"][row] == pytest.approx(o.g(eta), rel=1e-13)


@pytest.mark.parametrize("row", [0, 100, 255])
def test_energy_cutoff_fraction(orc_tables, golden, row):
    # the photons below xi_min carry 1e-9 of the spectrum's energy (Sec. 3), checked with QUADPACK
    si = pytest.importorskip("scipy.integrate")
    eta = eta_nodes(orc_tables)[row]
    xmin = 1 / (1 + math.exp(-orc_tables.a["zeta_lo"][row]))
    F = lambda s: 3 * s * s * o.F(eta, 0.5 * eta * s**3)  # F dxi in s = xi^{1/3}
    below = si.quad(F, 0, xmin ** (1 / 3), epsabs=0, epsrel=1e-12, limit=200)[0]
    total = si.quad(F, 0, 1, epsabs=0, epsrel=1e-12, limit=500, points=[0.01, 0.05, 0.2, 0.5])[0]
    assert below / total == pytest.approx(golden["energy_cut"]["value"], rel=1e-8)


@pytest.mark.parametrize("row", [10, 128, 240])
def test_P_row_against_quadpack(orc_tables, row):
    si = pytest.importorskip("scipy.integrate")
    eta = eta_nodes(orc_tables)[row]
    p = orc_tables.params
    zlo, zhi = orc_tables.a["zeta_lo"][row], orc_tables.a["zeta_hi"][row]
    h = math.exp(orc_tables.a["ln_h"][row])
    for j in (0, 50, 128, 200, 250):
        xi = 1 / (1 + math.exp(-(zlo + j * (zhi - zlo) / (p.n_xi - 1))))
        val = si.quad(lambda s: 3 * o.F(eta, 0.5 * eta * s**3) / s, 0, xi ** (1 / 3), epsabs=0, epsrel=1e-12,
                      limit=500)[0] / h
        assert orc_tables.a["P"][row, j] == pytest.approx(val, rel=1e-10)


def test_lookup_h_and_T_interpolation(orc_tables):
    # log-log linear interpolation: exact at nodes, small error between them
    nodes = eta_nodes(orc_tables)
    for i in (3, 77, 180):
        assert orc_tables.h(nodes[i]) == pytest.approx(math.exp(orc_tables.a["ln_h"][i]), rel=1e-14)
        mid = math.sqrt(nodes[i] * nodes[i + 1])
        assert orc_tables.h(mid) == pytest.approx(o.h(mid), rel=1e-4)
    # the curvature of ln T in ln chi (about 4/(3 chi)) bounds the error by 4/(3chi) d^2/8
    for chi, rel in ((0.05, 1e-2), (0.5, 1e-3), (5.0, 1e-4), (50.0, 1e-4)):
        assert orc_tables.T(chi) == pytest.approx(o.T(chi), rel=rel)
    assert orc_tables.T(0.5 * orc_tables.params.chi_min) == 0.0
    # above the table: chi^{-1/3} continuation of App. B
    big = 8 * orc_tables.params.chi_max
    assert orc_tables.T(big) == pytest.approx(o.T(orc_tables.params.chi_max) / 2, rel=1e-3)


def exact_xi_quantile(eta, U):
    """Invert the exact cumulative P_chi(xi) by bisection on quadrature (test-side reference)."""
    si = pytest.importorskip("scipy.integrate")
    h = o.h(eta)
    f = lambda s: 3 * o.F(eta, 0.5 * eta * s**3) / s
    lo, hi = 1e-16, 1.0
    for _ in range(60):
        mid = (lo * hi) ** 0.5 if hi / lo > 4 else 0.5 * (lo + hi)
        P = si.quad(f, 0, mid ** (1 / 3), epsabs=0, epsrel=1e-11, limit=500)[0] / h
        if P < U:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("eta", [1e-3, 0.7, 9.0])
def test_sample_xi_quantiles(orc_tables, eta):
    # inverse-CDF sampling of Sec. 3 against the exact quantile of p_chi; linear
    # interpolation between nodes about 4-10% apart in xi bounds the error to ~1%
    for U in (0.02, 0.2, 0.5, 0.8, 0.97, 0.999):
        xi = orc_tables.sample_xi(eta, U)
        assert xi == pytest.approx(exact_xi_quantile(eta, U), rel=0.01)
    assert orc_tables.sample_xi(eta, 1e-6) is None  # below the cut-off: ignored photon


@pytest.mark.parametrize("eta", [0.01, 1.0, 9.0, 55.0])
def test_sample_xi_mean_matches_power(orc_tables, eta):
    # E[xi] = int F dxi / h = 4 pi eta g / (3 sqrt3 h): the sampled photon energy times the
    # rate of eq. (rate_photons) reproduces the power P = P_c g(eta) of Sec. 2.1
    N = 200_000
    U = (np.arange(N) + 0.5) / N
    xs = np.array([orc_tables.sample_xi(eta, u) or 0.0 for u in U])
    exact = 4 * math.pi * eta * o.g(eta) / (3 * math.sqrt(3) * o.h(eta))
    assert xs.mean() == pytest.approx(exact, rel=3e-3)


@pytest.mark.parametrize("chi", [0.05, 0.7, 12.0])
def test_sample_f_symmetry_and_quantiles(orc_tables, chi):
    si = pytest.importorskip("scipy.integrate")
    k = o.k_norm(chi)
    for U in (0.03, 0.25, 0.45, 0.5, 0.7, 0.96):
        f = orc_tables.sample_f(chi, U)
        assert f + orc_tables.sample_f(chi, 1 - U) == pytest.approx(1.0, abs=1e-12)
        # exact CDF at the sampled f
        cdf = si.quad(lambda x: o.pf_unnorm(x, chi), 0, f, epsabs=0, epsrel=1e-11, limit=300)[0] / k
        assert cdf == pytest.approx(U, abs=3e-3)


@pytest.mark.parametrize("row", [0, 77, 200, 255])
def test_sample_xi_inverts_the_table_at_its_nodes(orc_tables, row):
    # whatever the interpolation between nodes, an inverse CDF taken at a node's tabulated
    # probability returns that node: P(xi_j) -> xi_j on the row's own eta (both halves: U <= 1/2
    # through P, U > 1/2 through Q).  A uniform U < 1 reaches complements Q >= 2^-53 only, so
    # the upper nodes are taken where 1 - Q is still Q to 1e-8.
    p = orc_tables.params
    eta = eta_nodes(orc_tables)[row]
    zlo, zhi = orc_tables.a["zeta_lo"][row], orc_tables.a["zeta_hi"][row]
    Qrow = orc_tables.a["Q"][row]
    top = int(np.nonzero(Qrow > 1e-8)[0].max())
    for j in (1, 40, 128, 200, top):
        xi_j = 1 / (1 + math.exp(-(zlo + j * (zhi - zlo) / (p.n_xi - 1))))
        P, Q = orc_tables.a["P"][row, j], Qrow[j]
        U = P if P <= 0.5 else 1.0 - Q
        assert orc_tables.sample_xi(eta, U) == pytest.approx(xi_j, rel=1e-9)


@pytest.mark.parametrize("row", [0, 90, 255])
def test_sample_f_inverts_the_table_at_its_nodes(orc_tables, row):
    # P_f at node f_j = j/(2(n_f - 1)) returns f_j for U = P_f/2 (lower half) and 1 - f_j for
    # U = 1 - P_f/2 (upper half, App. B's symmetry); nodes whose P_f is 0 or repeats its
    # predecessor (underflow at small chi, where pairs split almost evenly) are no inverse's image
    p = orc_tables.params
    chi = math.exp(math.log(p.chi_min) + row * (math.log(p.chi_max) - math.log(p.chi_min)) / (p.n_chi - 1))
    Pf = orc_tables.a["Pf"][row]
    nodes = [j for j in range(1, p.n_f - 1) if Pf[j] > 1e-12 and Pf[j] > Pf[j - 1]]
    assert len(nodes) > 10
    for j in nodes[:: max(1, len(nodes) // 6)]:
        f_j = 0.5 * j / (p.n_f - 1)
        V = Pf[j]
        assert orc_tables.sample_f(chi, 0.5 * V) == pytest.approx(f_j, rel=1e-9)
        if V > 1e-6:  # 1 - V/2 keeps V to 2^-53 absolute only
            assert orc_tables.sample_f(chi, 1.0 - 0.5 * V) == pytest.approx(1.0 - f_j, rel=1e-9)
