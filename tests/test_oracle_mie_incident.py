"""Pins for the oracle's Mie T-matrix (App. B) and initial-field coefficients
(App. A.2, App. C).  CPU only."""

import numpy as np
import pytest

from oracle import incident, mie, solve, svwf

K = 2 * np.pi / 550.0


@pytest.mark.parametrize("R,n", [(100.0, 1.52), (150.0, 1.5 + 0.001j), (130.0, 2.0), (60.0, 1.33 + 0.2j),
                                 (200.0, 1.45)])
def test_mie_matches_bohren_huffman(R, n):
    # Q_1l = -b_l, Q_2l = -a_l (Bohren & Huffman's Riccati-Bessel form)
    L = 6
    Q = mie.mie_q(L, K, R, n)
    a, b = mie.bohren_huffman_ab(L, K * R, n)
    assert np.allclose(Q[0], -b, rtol=1e-12, atol=1e-15)
    assert np.allclose(Q[1], -a, rtol=1e-12, atol=1e-15)


def _bhmie_log_derivative(lmax, x, m):
    """Mie a_l, b_l by the logarithmic-derivative method of Bohren & Huffman
    (their BHMIE program, written out here): D_l(mx) by downward recurrence
    D_{l-1} = l/z - 1/(D_l + l/z) from far above, Riccati-Bessel psi_l(x),
    chi_l(x) by upward recurrence from their closed forms (stable for l < x).
    It uses no library Bessel function of a complex argument, so it checks the
    oracle's complex-argument path at large size parameters independently."""
    z = m * x
    nstart = int(max(lmax, abs(z)) + 16 + 4 * abs(z) ** (1 / 3))
    D = [0j] * (nstart + 1)
    for n in range(nstart, 0, -1):
        D[n - 1] = n / z - 1.0 / (D[n] + n / z)
    psi = [np.sin(x), np.sin(x) / x - np.cos(x)]
    chi = [np.cos(x), np.cos(x) / x + np.sin(x)]
    for n in range(2, lmax + 1):
        psi.append((2 * n - 1) / x * psi[n - 1] - psi[n - 2])
        chi.append((2 * n - 1) / x * chi[n - 1] - chi[n - 2])
    a = np.zeros(lmax, dtype=complex)
    b = np.zeros(lmax, dtype=complex)
    for n in range(1, lmax + 1):
        xi_n, xi_m = psi[n] - 1j * chi[n], psi[n - 1] - 1j * chi[n - 1]
        fa = D[n] / m + n / x
        fb = m * D[n] + n / x
        a[n - 1] = (fa * psi[n] - psi[n - 1]) / (fa * xi_n - xi_m)
        b[n - 1] = (fb * psi[n] - psi[n - 1]) / (fb * xi_n - xi_m)
    return a, b


@pytest.mark.parametrize("x", [4.0, 10.0, 22.0, 30.0])
@pytest.mark.parametrize("n", [1.5 + 0.05j, 2.0 + 0.3j, 1.33 + 1e-3j, 1.7 + 0j])
def test_mie_large_size_parameters_vs_log_derivative_method(x, n):
    # Q_1l = -b_l, Q_2l = -a_l up to size parameter 30 with absorbing spheres
    L = 6
    Q = mie.mie_q(L, 1.0, x, n)
    a, b = _bhmie_log_derivative(L, x, n)
    assert np.allclose(Q[0], -b, rtol=1e-11, atol=1e-14)
    assert np.allclose(Q[1], -a, rtol=1e-11, atol=1e-14)


def test_gaussian_beam_rule_converged_far_from_the_axis():
    # the 128-node beta rule against 256 nodes at k rho ~ 100 from the beam
    # axis (the edge of the 10 000-sphere slab): agreement to 1e-13 of the
    # beam's peak coefficient
    k = K
    w = 2000.0
    pos = np.array([[8600.0, 300.0, 1500.0], [-5000.0, 7000.0, 400.0], [0.0, 0.0, 1000.0]])
    a128 = incident.gaussian_beam_coeffs(4, k, pos, w, (0.0, 0.0, 0.0), -np.pi / 2, n_beta=128)
    a256 = incident.gaussian_beam_coeffs(4, k, pos, w, (0.0, 0.0, 0.0), -np.pi / 2, n_beta=256)
    peak = np.max(np.abs(a256[2]))
    assert np.max(np.abs(a128 - a256)) < 1e-13 * peak


def test_mie_rayleigh_limit():
    # x -> 0: a_1 ~ -(2i/3) x^3 (m^2 - 1)/(m^2 + 2)
    n = 1.6 + 0.05j
    x = 1e-3
    Q = mie.mie_q(2, 1.0, x, n)
    a1 = -Q[1, 0]
    ref = -2j / 3 * x ** 3 * (n * n - 1) / (n * n + 2)
    assert abs(a1 - ref) < 1e-5 * abs(ref)


def test_lossless_sphere_has_no_absorption():
    # real n: Re(1/Q) = -1 for every Q, i.e. |Q + 1/2| = 1/2
    Q = mie.mie_q(5, K, 130.0, 1.52)
    assert np.allclose(np.real(1.0 / Q), -1.0, atol=1e-12)


@pytest.mark.parametrize("beta,alpha,pol", [(0.0, 0.0, 2), (0.0, 0.0, 1), (0.7, 1.1, 1), (2.3, -0.4, 2),
                                            (np.pi / 2, 0.3, 2)])
def test_plane_wave_expansion_identity(beta, alpha, pol):
    # sum_n a_n Psi^(1)_n(r - r_i) = E0 Phi_j(alpha, beta; r) near r_i (App. A.2)
    rng = np.random.default_rng(2)
    Lh = 25
    ri = np.array([[30.0, -20.0, 50.0]])
    pts = ri + rng.normal(size=(6, 3)) * 40.0
    a = incident.plane_wave_coeffs(Lh, K, ri, beta, alpha, pol)[0]
    E = svwf.field_expansion(1, a, Lh, K, pts, origin=ri[0])
    assert np.max(np.abs(E - svwf.pvwf(pol, alpha, beta, K, pts))) < 1e-12


def test_x_polarised_plane_wave_along_z():
    # beta = 0, alpha = 0, j = 2 is x-polarised: E = e_x e^{ikz}
    pts = np.array([[0.0, 0.0, 0.0], [10.0, 5.0, 70.0]])
    E = svwf.pvwf(2, 0.0, 0.0, K, pts)
    assert np.allclose(E[:, 0], np.exp(1j * K * pts[:, 2])) and np.allclose(E[:, 1:], 0)


def test_single_sphere_cross_sections_match_mie_series():
    # one sphere in a unit plane wave: b = T a;  C_ext, C_sca from the
    # project's normalisation equal the Mie series (2pi/k^2) sum (2l+1)(...)
    L = 8
    for R, n in [(100.0, 1.52), (150.0, 1.5 + 0.01j), (250.0, 1.33 + 0.3j)]:
        pos = np.zeros((1, 3))
        a = incident.plane_wave_coeffs(L, K, pos, 0.4, 0.9, 1)
        t = mie.t_diagonal(L, K, [R], [n])
        b = t * a
        aa, bb = mie.bohren_huffman_ab(L, K * R, n)
        ll = np.arange(1, L + 1)
        cext = 2 * np.pi / K ** 2 * np.sum((2 * ll + 1) * np.real(aa + bb))
        csca = 2 * np.pi / K ** 2 * np.sum((2 * ll + 1) * (np.abs(aa) ** 2 + np.abs(bb) ** 2))
        assert abs(solve.c_ext(K, a, b) - cext) < 1e-10 * cext
        assert abs(solve.c_sca_single(K, b) - csca) < 1e-10 * csca
        assert abs(solve.c_abs(K, t, b) - (cext - csca)) < 1e-9 * cext


def test_gaussian_beam_coefficients_reproduce_the_beam():
    # sum_n a_n Psi^(1)_n(r - r_i) equals E_in(r) of App. C computed by direct
    # 2D quadrature of the angular spectrum, near an off-axis sphere centre
    k = K
    w = 1500.0
    focus = np.array([40.0, -30.0, -200.0])
    ri = np.array([[350.0, 120.0, 300.0]])
    Lh = 16
    a = incident.gaussian_beam_coeffs(Lh, k, ri, w, focus, -np.pi / 2, n_beta=96)[0]
    rng = np.random.default_rng(9)
    pts = ri + rng.normal(size=(4, 3)) * 30.0
    E = svwf.field_expansion(1, a, Lh, k, pts, origin=ri[0])
    Ed = incident.gaussian_beam_field(k, w, focus, -np.pi / 2, pts, n_beta=96, n_alpha=96)
    assert np.max(np.abs(E - Ed)) < 1e-10 * np.max(np.abs(Ed))


def test_gaussian_beam_focus_and_profile():
    # for k w >> 1 the beam at its focus is ~ E0 e_x and its focal-plane
    # intensity profile ~ exp(-2 rho^2 / w^2) (paraxial limit, App. C)
    k = K
    w = 4000.0
    focus = np.zeros(3)
    pts = np.array([[0.0, 0.0, 0.0], [2000.0, 0.0, 0.0], [0.0, 3000.0, 0.0]])
    E = incident.gaussian_beam_field(k, w, focus, -np.pi / 2, pts, n_beta=80, n_alpha=64)
    assert abs(E[0, 0] - 1.0) < 2e-3 and np.max(np.abs(E[0, 1:])) < 2e-3
    rho2 = np.sum(pts[1:, :2] ** 2, axis=1)
    assert np.allclose(np.abs(E[1:, 0]), np.exp(-rho2 / w ** 2), atol=5e-3)
