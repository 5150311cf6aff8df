"""Initial-field SVWF coefficients a_in (App. A.2 PVWF->SVWF, App. C), FP64.

Test infrastructure only (see the package docstring).

Transformation operator (App. A.2, Eq. for B):
  B_nj(beta) = -1/i^{l+1} * 1/sqrt(2l(l+1)) * (i delta_j1 + delta_j2)
               * ( delta_{tau j} tau_l^|m|(beta) + (1 - delta_{tau j}) m pi_l^|m|(beta) )
and B^dagger_nj has every explicit i replaced by -i (so 1/i^{l+1} -> 1/(-i)^{l+1}).
The Gaussian-beam formulas write both B^dagger_{jn} and B^dagger_{nj}; both are
read as this one object.

Plane wave E_in(r) = E0 Phi_j(alpha, beta; r): expanding about r_i with the
PVWF->SVWF transform gives  a^i_n = 4 E0 e^{i k.r_i} e^{-i m alpha} B^dagger_nj(beta).

Gaussian beam (App. C): the paraxial-polarisation angular-spectrum beam
  E_in(r) = E0 k^2 w^2/(4 pi) sum_j int_0^{pi/2} dbeta sin(b) cos(b) exp(-w^2 k^2 sin^2(b)/4)
            int_0^{2pi} dalpha [e^{i(a-aG)}(d_j1 - i d_j2)/2 + e^{-i(a-aG)}(d_j1 + i d_j2)/2]
            Phi_j(alpha, beta; r - r_G)
(the printed "+" between the two exponentials of e^{ik.(r_i - r_G)} is read as
a product).  Its coefficients about r_i are

  a^i_n = E0 k^2 w^2/pi sum_j int_0^{pi/2} dbeta sin cos exp(-w^2k^2 sin^2/4 + i k z_Gi cos)
          B^dagger_nj(beta) I_jn(beta),
  I_jn(beta) = int_0^{2pi} dalpha [...] e^{-i m alpha} e^{i k rho_Gi sin(b) cos(alpha - phi_Gi)}.

The oracle evaluates I_jn by direct trapezoidal quadrature in alpha (exact to
rounding for these trigonometric integrands once the rule has enough points),
not by the Bessel-function closed form, and the beta integral by
Gauss-Legendre quadrature on [0, beta_max] where beta_max cuts the Gaussian
factor below 1e-17 (or pi/2).
"""

import numpy as np

from . import special as sf
from .svwf import multi_indices


def b_transform(tau, l, m, j, beta, dagger=False):
    """B_nj(beta) (or B^dagger_nj) for n = (tau, l, m), j in {1, 2}."""
    beta = np.asarray(beta, dtype=float)
    ct, st = np.cos(beta), np.sin(beta)
    iu = -1j if dagger else 1j
    pref = -1.0 / iu ** (l + 1) / np.sqrt(2.0 * l * (l + 1)) * (iu if j == 1 else 1.0)
    if tau == j:
        ang = sf.legendre_tau(l, abs(m), ct, st)
    else:
        ang = m * sf.legendre_pi(l, abs(m), ct, st)
    return pref * ang


def plane_wave_coeffs(lmax, k, positions, beta, alpha, pol, E0=1.0):
    """a_in for E_in = E0 Phi_pol(alpha, beta; r), shape (N, nmax)."""
    pos = np.atleast_2d(np.asarray(positions, dtype=float))
    kvec = k * np.array([np.sin(beta) * np.cos(alpha), np.sin(beta) * np.sin(alpha), np.cos(beta)])
    eikr = np.exp(1j * pos @ kvec)
    idx = multi_indices(lmax)
    out = np.zeros((pos.shape[0], len(idx)), dtype=complex)
    for n, (tau, l, m) in enumerate(idx):
        out[:, n] = 4.0 * E0 * eikr * np.exp(-1j * m * alpha) * b_transform(tau, l, m, pol, beta, dagger=True)
    return out


def gaussian_beta_max(k, w):
    """Upper beta limit: exp(-w^2 k^2 sin^2(beta)/4) < 1e-17 beyond it."""
    a = (w * k) ** 2 / 4.0
    s2 = 39.2 / a
    return np.pi / 2 if s2 >= 1.0 else float(np.arcsin(np.sqrt(s2)))


def gaussian_beam_coeffs(lmax, k, positions, w, focus, alpha_G, E0=1.0, n_beta=256, n_alpha=None):
    """a_in of the Gaussian beam of App. C about each sphere centre, (N, nmax).

    ``focus`` = r_G, ``alpha_G`` sets E_0 = (-sin aG e_x + cos aG e_y) E0.
    """
    pos = np.atleast_2d(np.asarray(positions, dtype=float))
    rel = pos - np.asarray(focus, dtype=float)[None, :]
    rho = np.hypot(rel[:, 0], rel[:, 1])
    phiG = np.arctan2(rel[:, 1], rel[:, 0])
    zG = rel[:, 2]
    bmax = gaussian_beta_max(k, w)
    xg, wg = np.polynomial.legendre.leggauss(n_beta)
    beta = 0.5 * bmax * (xg + 1.0)
    wb = 0.5 * bmax * wg
    krmax = k * (np.max(rho) if rho.size else 0.0)
    if n_alpha is None:
        n_alpha = int(2 * (krmax + lmax + 40))
    alpha = 2.0 * np.pi * np.arange(n_alpha) / n_alpha
    wa = 2.0 * np.pi / n_alpha
    sb, cb = np.sin(beta), np.cos(beta)
    gauss = sb * cb * np.exp(-(w * k * sb) ** 2 / 4.0)               # (nb,)
    idx = multi_indices(lmax)
    out = np.zeros((pos.shape[0], len(idx)), dtype=complex)
    ea = np.exp(1j * (alpha - alpha_G))
    for i in range(pos.shape[0]):
        # e^{i k rho sin(b) cos(a - phi)}: (nb, na)
        plane = np.exp(1j * k * rho[i] * sb[:, None] * np.cos(alpha[None, :] - phiG[i]))
        zfac = np.exp(1j * k * zG[i] * cb)                            # (nb,)
        for j in (1, 2):
            # e^{i(a-aG)}(d_j1 - i d_j2)/2 + e^{-i(a-aG)}(d_j1 + i d_j2)/2
            if j == 1:
                polw = (ea + 1.0 / ea) / 2.0
            else:
                polw = (-1j * ea + 1j / ea) / 2.0
            for n, (tau, l, m) in enumerate(idx):
                I = (plane * (polw * np.exp(-1j * m * alpha))[None, :]).sum(axis=1) * wa  # (nb,)
                Bd = b_transform(tau, l, m, j, beta, dagger=True)
                out[i, n] += E0 * (k * w) ** 2 / np.pi * np.sum(wb * gauss * zfac * Bd * I)
    return out


def gaussian_beam_field(k, w, focus, alpha_G, r, E0=1.0, n_beta=256, n_alpha=256):
    """E_in(r) of App. C by direct 2D quadrature of its angular spectrum."""
    r = np.atleast_2d(np.asarray(r, dtype=float)) - np.asarray(focus, dtype=float)[None, :]
    bmax = gaussian_beta_max(k, w)
    xg, wg = np.polynomial.legendre.leggauss(n_beta)
    beta = 0.5 * bmax * (xg + 1.0)
    wb = 0.5 * bmax * wg
    alpha = 2.0 * np.pi * np.arange(n_alpha) / n_alpha
    wa = 2.0 * np.pi / n_alpha
    out = np.zeros((r.shape[0], 3), dtype=complex)
    for ib, b in enumerate(beta):
        g = np.sin(b) * np.cos(b) * np.exp(-(w * k * np.sin(b)) ** 2 / 4.0)
        if g == 0.0:
            continue
        for a in alpha:
            d = a - alpha_G
            c1 = np.cos(d)          # (e^{id} + e^{-id})/2
            c2 = np.sin(d)          # (-i e^{id} + i e^{-id})/2
            kvec = k * np.array([np.sin(b) * np.cos(a), np.sin(b) * np.sin(a), np.cos(b)])
            ph = np.exp(1j * r @ kvec)
            ca, sa, cbb, sbb = np.cos(a), np.sin(a), np.cos(b), np.sin(b)
            e_a = np.array([-sa, ca, 0.0])
            e_b = np.array([cbb * ca, cbb * sa, -sbb])
            out += (wb[ib] * wa * g) * ph[:, None] * (c1 * e_a + c2 * e_b)[None, :]
    return E0 * (k * w) ** 2 / (4.0 * np.pi) * out
