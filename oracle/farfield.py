"""Plane-wave amplitude of the scattered field (App. D), FP64.

Test infrastructure only (see the package docstring).

Inserting the SVWF->PVWF transform (App. A.2) into the scattered field
E_scat = sum_i sum_n b^i_n Psi^(3)_n(r - r_i) (Sec. 2.1) and using
Phi_j(alpha, beta; r - r_i) = e^{-i k.r_i} Phi_j(alpha, beta; r) gives the
plane-wave expansion E = sum_j int dalpha int dbeta sin(beta) g_j Phi_j with

  g_j(alpha, beta) = 1/(2 pi) sum_i e^{-i k(alpha,beta).r_i} sum_n B_nj(beta) e^{i m alpha} b^i_n

(beta in [0, pi/2] for the forward half space, [pi/2, pi] backward).  The
radiant intensity is I_j = 2 pi^2/(omega k mu0) |g_j|^2 (App. D).
"""

import numpy as np

from .incident import b_transform
from .svwf import multi_indices


def farfield_amplitude(lmax, k, positions, b, dirs):
    """g_j for each direction; ``dirs`` (Nd, 2) = (beta, alpha).  Returns (Nd, 2)."""
    pos = np.atleast_2d(np.asarray(positions, dtype=float))
    bb = np.asarray(b).reshape(pos.shape[0], -1)
    dirs = np.atleast_2d(np.asarray(dirs, dtype=float))
    idx = multi_indices(lmax)
    out = np.zeros((dirs.shape[0], 2), dtype=complex)
    for q, (beta, alpha) in enumerate(dirs):
        kvec = k * np.array([np.sin(beta) * np.cos(alpha), np.sin(beta) * np.sin(alpha), np.cos(beta)])
        ph = np.exp(-1j * pos @ kvec)                        # (N,)
        for j in (1, 2):
            coef = np.array([b_transform(tau, l, m, j, beta) * np.exp(1j * m * alpha)
                             for (tau, l, m) in idx], dtype=complex)   # (nmax,)
            out[q, j - 1] = np.sum(ph * (bb @ coef)) / (2.0 * np.pi)
    return out


def c_sca_quadrature(lmax, k, positions, b, n_beta=64, n_alpha=128, E0=1.0):
    """Scattering cross section from |g|^2 integrated over all directions:
    C_sca = (4 pi^2 / k^2) int dOmega sum_j |g_j|^2 / |E0|^2.

    (Stationary phase on the plane-wave expansion gives
    E_scat ~ -2 pi i e^{ikr}/(kr) sum_j g_j e_j at large r.)
    """
    xg, wg = np.polynomial.legendre.leggauss(n_beta)
    beta = np.arccos(-xg)                 # cos(beta) = -xg  -> beta in (0, pi)
    alpha = 2.0 * np.pi * np.arange(n_alpha) / n_alpha
    B, A = np.meshgrid(beta, alpha, indexing="ij")
    dirs = np.stack([B.ravel(), A.ravel()], axis=1)
    g = farfield_amplitude(lmax, k, positions, b, dirs)
    I = np.sum(np.abs(g) ** 2, axis=1).reshape(n_beta, n_alpha)
    total = np.sum(wg[:, None] * I) * (2.0 * np.pi / n_alpha)
    return float(4.0 * np.pi ** 2 / k ** 2 * total / abs(E0) ** 2)


def s11_azimuthal(lmax, k, positions, b_te, b_tm, betas, n_alpha=64):
    """S11(beta) as in the phase-matrix comparison of Sec. 4: the scattered
    intensity sum_j |g_j|^2 averaged over the azimuth (trapezoid, n_alpha
    nodes) and over a TE and a TM run, unnormalised."""
    betas = np.atleast_1d(np.asarray(betas, dtype=float))
    alpha = 2.0 * np.pi * np.arange(n_alpha) / n_alpha
    B, A = np.meshgrid(betas, alpha, indexing="ij")
    dirs = np.stack([B.ravel(), A.ravel()], axis=1)
    out = np.zeros(betas.size)
    for b in (b_te, b_tm):
        g = farfield_amplitude(lmax, k, positions, b, dirs)
        out += np.sum(np.abs(g) ** 2, axis=1).reshape(betas.size, n_alpha).mean(axis=1)
    return 0.5 * out
