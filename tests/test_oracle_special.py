"""Pins of the oracle's special functions and emissivities (App. A, App. B) against closed
forms, library routines and brute-force quadrature.  CPU only."""
import math

import numpy as np
import pytest

import oracle as o

GAMMA = math.gamma


# ------------------------------------------------------------------ Bessel functions
@pytest.mark.parametrize("x", [1e-8, 1e-3, 0.1, 1.0, 7.5, 40.0, 300.0])
def test_besselk_half_order_closed_form(x):
    # K_{1/2}(x) = sqrt(pi/(2x)) e^{-x}, K_{3/2}(x) = sqrt(pi/(2x)) e^{-x} (1 + 1/x)
    k12 = math.sqrt(math.pi / (2 * x)) * math.exp(-x)
    assert o.besselk(0.5, x) == pytest.approx(k12, rel=1e-13)
    assert o.besselk(1.5, x) == pytest.approx(k12 * (1 + 1 / x), rel=1e-13)


@pytest.mark.parametrize("y", [1e-8, 1e-3, 0.3, 2.0, 25.0])
def test_besselk_integral_half_order_closed_form(y):
    # int_y^inf K_{1/2} = sqrt(pi/2) Gamma(1/2, y) = (pi/sqrt2) erfc(sqrt y)
    ref = math.pi / math.sqrt(2) * math.erfc(math.sqrt(y))
    assert o.besselk_int(0.5, y) == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("nu", [1 / 3, 2 / 3, 5 / 3])
def test_besselk_against_scipy(nu):
    sp = pytest.importorskip("scipy.special")
    for x in np.geomspace(1e-10, 600, 37):
        assert o.besselk(nu, x) == pytest.approx(sp.kv(nu, x), rel=2e-13)


@pytest.mark.parametrize("y", [1e-9, 1e-4, 0.05, 0.7, 3.0, 20.0])
def test_ki53_recurrence_identity(y):
    # K'_{2/3} = -(K_{1/3} + K_{5/3})/2  =>  Ki_{5/3}(y) = 2 K_{2/3}(y) - Ki_{1/3}(y)
    lhs = o.besselk_int(5 / 3, y)
    rhs = 2 * o.besselk(2 / 3, y) - o.besselk_int(1 / 3, y)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_ki13_total_integral():
    # int_0^inf K_nu = pi / (2 cos(nu pi/2)); for nu = 1/3 this is pi/sqrt3
    assert o.besselk_int(1 / 3, 1e-14) == pytest.approx(math.pi / math.sqrt(3), rel=1e-4)


# ------------------------------------------------------------------ Philox4x64-10
@pytest.mark.parametrize("ctr,key", [([0, 0, 0, 0], [0, 0]), ([5, 0, 0, 0], [5, 7]),
                                     ([2**64 - 1, 3, 9, 2], [123456789, 987654321]),
                                     ([17, 2**63, 2, 1], [1, 2**64 - 1])])
def test_philox_against_numpy(ctr, key):
    # numpy's Philox (4x64, 10 rounds) first advances its counter, then emits one block.
    np_ = pytest.importorskip("numpy")
    prev = list(ctr)
    for i in range(4):  # decrement with borrow
        if prev[i] > 0:
            prev[i] -= 1
            break
        prev[i] = 2**64 - 1
    bg = np_.random.Philox(key=np_.array(key, dtype=np_.uint64), counter=np_.array(prev, dtype=np_.uint64))
    ref = [int(v) for v in bg.random_raw(4)]
    assert o.philox4x64(ctr, key) == ref


def test_u01_open_interval_and_uniform():
    assert 0.0 < o.u01(0) < 1e-15
    assert 1.0 - 1e-15 < o.u01(2**64 - 1) < 1.0
    us = np.array([o.u01(w) for blk in range(2000) for w in o.philox4x64([blk, 7, 2, 0], [3, 4])])
    assert abs(us.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(us))
    hist, _ = np.histogram(us, bins=16, range=(0, 1))
    chi2 = ((hist - len(us) / 16) ** 2 / (len(us) / 16)).sum()
    assert chi2 < 45  # 15 dof, p ~ 1e-4


# ------------------------------------------------------------------ F, h, g (App. A)
def test_F_zero_above_kinematic_limit():
    for eta in (0.1, 1.0, 10.0):
        assert o.F(eta, 0.5 * eta) == 0.0
        assert o.F(eta, 0.6 * eta) == 0.0
        assert o.F(eta, 0.49 * eta) > 0.0


@pytest.mark.parametrize("yc", [0.01, 0.3, 1.0, 4.0])
def test_F_classical_limit(yc):
    # hbar -> 0 (eta -> 0 at fixed y_c = 4chi/(3 eta^2)): F -> y_c Ki_{5/3}(y_c)
    # the leading correction is O(eta y_c): the gap shrinks a hundredfold per hundredfold in eta
    for eta in (1e-3, 1e-5, 1e-7):
        chi = 0.75 * yc * eta * eta
        assert o.F(eta, chi) == pytest.approx(o.F_classical(eta, chi), rel=8 * eta * (1 + yc))


def test_h_classical_limit():
    # h0 = int_0^inf y Ki_{5/3}(y) dy/y ... = Gamma(1/6) Gamma(11/6) = 5 pi/3 (printed 5.24)
    h0 = GAMMA(1 / 6) * GAMMA(11 / 6)
    assert h0 == pytest.approx(5 * math.pi / 3, rel=1e-14)
    assert o.h(1e-7) == pytest.approx(h0, rel=2e-6)
    # first quantum correction: 1 - h/h0 -> (8 sqrt3 / 15) eta
    for eta in (1e-5, 1e-6):
        assert (1 - o.h(eta) / h0) / eta == pytest.approx(8 * math.sqrt(3) / 15, rel=2e-3)


def test_h0_printed_value(golden):
    assert round(5 * math.pi / 3, 2) == golden["h0"]["value"]


def test_g_classical_limit():
    assert o.g(1e-7) == pytest.approx(1.0, abs=1e-5)
    # power correction: 1 - g -> (55 sqrt3/16) eta - 48 eta^2
    for eta in (1e-4, 1e-5):
        assert (1 - o.g(eta)) / eta == pytest.approx(55 * math.sqrt(3) / 16 - 48 * eta, rel=2e-3)


def test_g_fit_of_section_2_1(golden):
    # the fit of Sec. 2.1 agrees with the quadrature to about a percent over the table range
    for eta in np.geomspace(1e-4, 1e2, 25):
        assert o.g(eta) == pytest.approx(o.g_fit(eta), rel=0.015)
    assert o.g(1.0) == pytest.approx(golden["g_at_eta_1"]["value"], abs=0.02)


def test_h_g_bruteforce_quadpack():
    # brute force with a different integrator (QUADPACK) and library Bessel functions.
    # Ki_{5/3} = 2 K_{2/3} - Ki_{1/3} (from K'_{2/3} = -(K_{1/3}+K_{5/3})/2), with
    # Ki_{1/3}(y) = pi/sqrt3 - int_0^y K_{1/3} below y = 1; h and g in s = xi^{1/3}.
    sp = pytest.importorskip("scipy.special")
    si = pytest.importorskip("scipy.integrate")

    def ki13(y):
        if y < 1:
            return math.pi / math.sqrt(3) - si.quad(lambda t: sp.kv(1 / 3, t), 0, y, epsabs=0, epsrel=1e-13,
                                                    limit=200)[0]
        return si.quad(lambda t: sp.kv(1 / 3, t), y, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]

    def F(eta, s):
        xi = s**3
        omx = (1 - s) * (1 + s + s * s)
        if omx <= 0:
            return 0.0
        y = 2 * xi / (3 * eta * omx)
        if y > 700:
            return 0.0
        return xi * xi * y * sp.kv(2 / 3, y) + omx * y * (2 * sp.kv(2 / 3, y) - ki13(y))

    for eta in (0.5, 9.0):
        kw = dict(epsabs=0, epsrel=1e-12, limit=500, points=[0.05, 0.2, 0.5])
        h_ref = si.quad(lambda s: 3 * F(eta, s) / s, 0, 1, **kw)[0]
        G = si.quad(lambda s: 3 * s * s * F(eta, s), 0, 1, **kw)[0]
        g_ref = 3 * math.sqrt(3) / (4 * math.pi * eta) * G
        assert o.h(eta) == pytest.approx(h_ref, rel=1e-12)
        assert o.g(eta) == pytest.approx(g_ref, rel=1e-12)


# ------------------------------------------------------------------ T and p_f (App. B)
def test_T_maximum(golden):
    chis = np.geomspace(1, 50, 300)
    Ts = np.array([o.T(c) for c in chis])
    assert Ts.max() == pytest.approx(golden["max_T"]["value"], abs=0.005)
    assert 4 < chis[Ts.argmax()] < 10


def test_T_large_chi_power_law():
    # K_{1/3}(x) ~ Gamma(1/3)/2 (2/x)^{1/3}:  chi^{1/3} T -> 0.04 Gamma(1/3)^2 3^{2/3}
    lim = 0.04 * GAMMA(1 / 3) ** 2 * 3 ** (2 / 3)
    assert o.T(1e6) * 1e6 ** (1 / 3) == pytest.approx(lim, rel=1e-3)


def test_T_small_chi_exponent():
    # the formula of App. B gives T ~ exp(-4/(3 chi)) (the printed text says exp(-2/(3chi));
    # the formula governs): 0.16 (pi/(2x)) e^{-2x}/chi, x = 2/(3chi), to O(chi)
    for chi in (0.01, 0.003):
        x = 2 / (3 * chi)
        asym = 0.16 * (math.pi / (2 * x)) * math.exp(-2 * x) / chi
        assert o.T(chi) == pytest.approx(asym, rel=0.25 * chi * 10)


def test_pf_symmetry_and_normalisation():
    for chi in (0.1, 1.0, 10.0, 100.0):
        for f in (0.01, 0.1, 0.3, 0.45):
            assert o.pf_unnorm(f, chi) == pytest.approx(o.pf_unnorm(1 - f, chi), rel=1e-13)
    si = pytest.importorskip("scipy.integrate")
    for chi in (0.1, 1.0, 10.0):
        ref, _ = si.quad(lambda f: o.pf_unnorm(f, chi), 0, 1, epsabs=0, epsrel=1e-12, limit=200)
        assert o.k_norm(chi) == pytest.approx(ref, rel=1e-10)


def test_pf_shape_limits():
    # chi << 1: sharply peaked at f = 1/2; chi >> 1: peaked near the ends (App. B)
    assert o.pf_unnorm(0.5, 0.1) > 50 * o.pf_unnorm(0.2, 0.1)
    assert o.pf_unnorm(0.05, 100.0) > o.pf_unnorm(0.5, 100.0)
