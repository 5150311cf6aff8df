"""Pins for the oracle's special functions (App. A.1/A.2) against closed forms,
identities and an independent library.  CPU only."""

import numpy as np
import pytest
import scipy.special as sps
from fractions import Fraction
from math import factorial, sqrt

from oracle import special as sf


X = np.array([0.3, 0.9, 1.7, 2.28, 5.0, 13.7, 47.0, 230.0])


def test_h0_h1_closed_forms():
    # h_0 = -i e^{ix}/x ; j_0 = sin x / x ; y_0 = -cos x / x
    assert np.allclose(sf.sph_h1(0, X), -1j * np.exp(1j * X) / X, rtol=1e-14, atol=0)
    assert np.allclose(sf.sph_j(0, X), np.sin(X) / X, rtol=1e-13, atol=1e-16)
    assert np.allclose(sf.sph_y(0, X), -np.cos(X) / X, rtol=1e-13, atol=1e-16)
    # h_1 = -e^{ix}(x + i)/x^2
    assert np.allclose(sf.sph_h1(1, X), -np.exp(1j * X) * (X + 1j) / X ** 2, rtol=1e-13)


@pytest.mark.parametrize("l", range(0, 11))
def test_hankel_matches_finite_closed_form(l):
    assert np.allclose(sf.sph_h1(l, X), sf.sph_h1_closed(l, X), rtol=1e-11, atol=0)


@pytest.mark.parametrize("l", range(1, 11))
def test_wronskian(l):
    # j_l y_{l-1} - j_{l-1} y_l = 1/x^2
    w = sf.sph_j(l, X) * sf.sph_y(l - 1, X) - sf.sph_j(l - 1, X) * sf.sph_y(l, X)
    assert np.allclose(w, 1.0 / X ** 2, rtol=1e-10)


@pytest.mark.parametrize("z", [1.3, 2.7 + 0.01j, 4.1 + 0.3j])
def test_riccati_derivative_by_finite_difference(z):
    h = 1e-6
    for l in range(1, 6):
        fd = ((z + h) * sf.sph_j(l, z + h) - (z - h) * sf.sph_j(l, z - h)) / (2 * h)
        assert abs(sf.dxxj(l, z) - fd) < 1e-8
        if np.isreal(z):
            x = float(np.real(z))
            fdh = ((x + h) * sf.sph_h1(l, x + h) - (x - h) * sf.sph_h1(l, x - h)) / (2 * h)
            assert abs(sf.dxxh(l, x) - fdh) < 1e-7 * abs(fdh)


def test_legendre_normalisation_and_orthogonality():
    xg, wg = np.polynomial.legendre.leggauss(80)
    ct, st = xg, np.sqrt(1 - xg ** 2)
    for m in range(0, 8):
        for l in range(m, 12):
            p = sf.legendre_p(l, m, ct, st)
            assert abs(np.sum(wg * p * p) - 1.0) < 1e-12
            if l + 1 < 12 and l + 1 >= m:
                q = sf.legendre_p(l + 1, m, ct, st)
                assert abs(np.sum(wg * p * q)) < 1e-12


def test_legendre_against_scipy_lpmv():
    # scipy's lpmv carries the Condon-Shortley phase (-1)^m; ours does not.
    t = np.linspace(0.01, np.pi - 0.01, 17)
    ct, st = np.cos(t), np.sin(t)
    for l in range(0, 10):
        for m in range(0, l + 1):
            ref = (-1) ** m * sps.lpmv(m, l, ct) * sqrt((2 * l + 1) / 2 * factorial(l - m) / factorial(l + m))
            assert np.allclose(sf.legendre_p(l, m, ct, st), ref, rtol=1e-11, atol=1e-13)


def test_pi_tau_definitions():
    t = np.linspace(0.05, np.pi - 0.05, 13)
    ct, st = np.cos(t), np.sin(t)
    h = 1e-6
    for l in range(1, 9):
        for m in range(0, l + 1):
            P = sf.legendre_p(l, m, ct, st)
            if m > 0:
                assert np.allclose(sf.legendre_pi(l, m, ct, st) * st, P, rtol=1e-12, atol=1e-14)
            fd = (sf.legendre_p(l, m, np.cos(t + h), np.sin(t + h))
                  - sf.legendre_p(l, m, np.cos(t - h), np.sin(t - h))) / (2 * h)
            assert np.allclose(sf.legendre_tau(l, m, ct, st), fd, atol=1e-7)


def test_pi_tau_at_the_pole():
    # finite limits at theta = 0: pi_l^1(0) = tau_l^1(0) = N_l1 l(l+1)/2, others 0
    for l in range(1, 9):
        nl1 = sqrt((2 * l + 1) / 2 / (l * (l + 1)))
        assert abs(sf.legendre_pi(l, 1, 1.0, 0.0) - nl1 * l * (l + 1) / 2) < 1e-12
        assert abs(sf.legendre_tau(l, 1, 1.0, 0.0) - nl1 * l * (l + 1) / 2) < 1e-12
        for m in (0, 2, 3):
            if m <= l:
                assert abs(sf.legendre_pi(l, m, 1.0, 0.0)) < 1e-14
                assert abs(sf.legendre_tau(l, m, 1.0, 0.0)) < 1e-14


def test_wigner3j_exact_values():
    # textbook values
    assert abs(sf.wigner3j(1, 1, 0, 0, 0, 0) - (-1 / sqrt(3))) < 1e-15
    assert abs(sf.wigner3j(1, 1, 2, 0, 0, 0) - sqrt(2 / 15)) < 1e-15
    assert abs(sf.wigner3j(1, 1, 1, 1, -1, 0) - 1 / sqrt(6)) < 1e-15
    assert abs(sf.wigner3j(2, 2, 2, 0, 0, 0) - (-sqrt(2 / 35))) < 1e-15
    # odd sum with zero m's vanishes; selection rules
    assert sf.wigner3j(1, 1, 1, 0, 0, 0) == 0.0
    assert sf.wigner3j(2, 1, 4, 0, 0, 0) == 0.0
    assert sf.wigner3j(2, 2, 2, 1, 1, 0) == 0.0
    sign, sq = sf.wigner3j_sq_signed(3, 2, 1, 1, -1, 0)
    assert isinstance(sq, Fraction)


def test_wigner3j_orthogonality():
    # sum_{j3, m3} (2 j3 + 1) (j1 j2 j3; m1 m2 m3)^2 = 1
    for j1, j2 in [(1, 1), (2, 3), (4, 4), (5, 3)]:
        for m1 in range(-j1, j1 + 1):
            for m2 in range(-j2, j2 + 1):
                s = sum((2 * j3 + 1) * sf.wigner3j(j1, j2, j3, m1, m2, -m1 - m2) ** 2
                        for j3 in range(abs(j1 - j2), j1 + j2 + 1))
                assert abs(s - 1.0) < 1e-13


def test_wigner3j_against_sympy():
    wig = pytest.importorskip("sympy.physics.wigner")
    rng = np.random.default_rng(5)
    for _ in range(60):
        j1, j2 = rng.integers(0, 6, 2)
        j3 = rng.integers(abs(j1 - j2), j1 + j2 + 1)
        m1 = rng.integers(-j1, j1 + 1)
        m2 = rng.integers(-j2, j2 + 1)
        ref = float(wig.wigner_3j(int(j1), int(j2), int(j3), int(m1), int(m2), int(-m1 - m2)))
        assert abs(sf.wigner3j(int(j1), int(j2), int(j3), int(m1), int(m2), int(-m1 - m2)) - ref) < 1e-14
