"""Reflected and transmitted power of a Gaussian-beam simulation (App. D; the
reflectivity / transmittivity figures of Sec. 4), FP64.

Test infrastructure only (see the package docstring).

A field given as a plane-wave expansion E = sum_j int dalpha int dbeta
sin(beta) g_j(alpha, beta) Phi_j carries the flux
    P = C sum_j int dalpha int dbeta sin(beta) |g_j|^2,   C = 2 pi^2/(omega k mu0)
(App. D).  The Gaussian beam's amplitude (App. D) is
    g_in,j = E0 k^2 w^2/(4 pi) cos(b) exp(-w^2 k^2 sin^2(b)/4) e^{-i k.r_G}
             x (cos(a - a_G) for j = 1, sin(a - a_G) for j = 2),   b in [0, pi/2]
(the printed form is the a_G = 0 case), and its power is
    P_in = |E0|^2 pi k^3 w^4/(4 omega mu0) int_0^{pi/2} sin b cos^2 b exp(-w^2 k^2 sin^2(b)/2) db.
Transmitted power: the forward hemisphere (b < pi/2) of |g_in + g_sca|^2,
reflected power: the backward hemisphere of |g_sca|^2; R = P_back/P_in and
T = P_fwd/P_in (C cancels).  g_sca is the far-field amplitude of App. D.
Quadrature: Gauss-Legendre in beta on each hemisphere, trapezoid in alpha.
"""

import numpy as np

from .farfield import farfield_amplitude


def gaussian_amplitude(k, w, focus, alpha_G, dirs, E0=1.0):
    """g_in,j of the Gaussian beam at directions dirs (Nd, 2) = (beta, alpha); (Nd, 2)."""
    dirs = np.atleast_2d(np.asarray(dirs, dtype=float))
    b, a = dirs[:, 0], dirs[:, 1]
    kvec = k * np.stack([np.sin(b) * np.cos(a), np.sin(b) * np.sin(a), np.cos(b)], axis=1)
    ph = np.exp(-1j * kvec @ np.asarray(focus, dtype=float))
    amp = E0 * k ** 2 * w ** 2 / (4.0 * np.pi) * np.cos(b) * np.exp(-(w * k * np.sin(b)) ** 2 / 4.0) * ph
    amp = np.where(b <= np.pi / 2, amp, 0.0)
    return np.stack([amp * np.cos(a - alpha_G), amp * np.sin(a - alpha_G)], axis=1)


def gaussian_power_over_C(k, w, E0=1.0, n=4000):
    """P_in / C from the 1D integral of App. D (Gauss-Legendre with n nodes)."""
    x, wt = np.polynomial.legendre.leggauss(n)
    b = 0.25 * np.pi * (x + 1.0)
    f = np.sin(b) * np.cos(b) ** 2 * np.exp(-(w * k * np.sin(b)) ** 2 / 2.0)
    integral = 0.25 * np.pi * np.sum(wt * f)
    # C^-1 P_in = |E0|^2 (k^2 w^2/(4 pi))^2 * 2 pi * integral
    return abs(E0) ** 2 * (k ** 2 * w ** 2 / (4.0 * np.pi)) ** 2 * 2.0 * np.pi * integral


def hemisphere_rule(n_beta, n_alpha, forward):
    """Directions (n_beta * n_alpha, 2) and weights sin(beta) dbeta dalpha."""
    x, wt = np.polynomial.legendre.leggauss(n_beta)
    lo, hi = (0.0, 0.5 * np.pi) if forward else (0.5 * np.pi, np.pi)
    beta = lo + 0.5 * (hi - lo) * (x + 1.0)
    wb = 0.5 * (hi - lo) * wt * np.sin(beta)
    alpha = 2.0 * np.pi * np.arange(n_alpha) / n_alpha
    B, A = np.meshgrid(beta, alpha, indexing="ij")
    W = np.broadcast_to(wb[:, None] * (2.0 * np.pi / n_alpha), B.shape)
    return np.stack([B.ravel(), A.ravel()], axis=1), W.ravel()


def reflect_transmit(lmax, k, positions, b, w, focus, alpha_G, E0=1.0, n_beta=128, n_alpha=128):
    """(R, T) of the scattered coefficients b (N, nmax) under the Gaussian beam."""
    p_in = gaussian_power_over_C(k, w, E0)
    df, wf = hemisphere_rule(n_beta, n_alpha, True)
    db, wbk = hemisphere_rule(n_beta, n_alpha, False)
    gf = farfield_amplitude(lmax, k, positions, b, df) + gaussian_amplitude(k, w, focus, alpha_G, df, E0)
    gb = farfield_amplitude(lmax, k, positions, b, db)
    T = np.sum(wf * np.sum(np.abs(gf) ** 2, axis=1)) / p_in
    R = np.sum(wbk * np.sum(np.abs(gb) ** 2, axis=1)) / p_in
    return float(R), float(T)
