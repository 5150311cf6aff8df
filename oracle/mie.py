"""T-matrix of a sphere (App. B), FP64.

Test infrastructure only (see the package docstring).

T^i_{nn'} = Q^i_{tau l} delta_{tau tau'} delta_{l l'} delta_{m m'} with (App. B)

  Q_1l = [ j_l(x) d(y j_l(y)) - j_l(y) d(x j_l(x)) ] / [ j_l(y) d(x h_l(x)) - h_l(x) d(y j_l(y)) ]
  Q_2l = [ k^2 j_l(x) d(y j_l(y)) - k_i^2 j_l(y) d(x j_l(x)) ]
         / [ k_i^2 j_l(y) d(x h_l(x)) - k^2 h_l(x) d(y j_l(y)) ]

with x = k R_i, y = k_i R_i and each derivative taken with respect to the
argument of its own bracket (the paper's subscript "d_{kR}" in the Q_1
denominator is read as d_{kR_i}).  k is the background wavenumber n0*k0 and
k_i = (n_i/n0) k (the paper writes k_i = n_i k with n0 = 1 in all its runs).
"""

import numpy as np

from . import special as sf


def mie_q(lmax, k, radius, n_rel):
    """Return Q of shape (2, lmax): Q[0, l-1] = Q_1l, Q[1, l-1] = Q_2l.

    ``k``: background wavenumber; ``n_rel``: n_i / n0 (complex allowed).
    """
    x = k * radius
    y = n_rel * k * radius
    ki2 = (n_rel * k) ** 2
    k2 = k * k
    Q = np.zeros((2, lmax), dtype=complex)
    for l in range(1, lmax + 1):
        jx = sf.sph_j(l, x)
        jy = sf.sph_j(l, y)
        hx = sf.sph_h1(l, x)
        djx = sf.dxxj(l, x)
        djy = sf.dxxj(l, y)
        dhx = sf.dxxh(l, x)
        Q[0, l - 1] = (jx * djy - jy * djx) / (jy * dhx - hx * djy)
        Q[1, l - 1] = (k2 * jx * djy - ki2 * jy * djx) / (ki2 * jy * dhx - k2 * hx * djy)
    return Q


def t_diagonal(lmax, k, radii, n_rel):
    """Diagonal of T for N spheres, shape (N, nmax) in coefficient order."""
    radii = np.atleast_1d(np.asarray(radii, dtype=float))
    n_rel = np.broadcast_to(np.asarray(n_rel, dtype=complex), radii.shape)
    nh = lmax * (lmax + 2)
    out = np.zeros((radii.size, 2 * nh), dtype=complex)
    for i in range(radii.size):
        Q = mie_q(lmax, k, radii[i], n_rel[i])
        for l in range(1, lmax + 1):
            for m in range(-l, l + 1):
                n = l * (l + 1) - 1 + m
                out[i, n] = Q[0, l - 1]
                out[i, n + nh] = Q[1, l - 1]
    return out


def bohren_huffman_ab(lmax, x, m_rel):
    """Mie a_l, b_l in Bohren & Huffman's form (psi/xi Riccati functions),
    an independent textbook route used only as a pin:
      a_l = [m psi_l(mx) psi_l'(x) - psi_l(x) psi_l'(mx)] / [m psi_l(mx) xi_l'(x) - xi_l(x) psi_l'(mx)]
      b_l = [psi_l(mx) psi_l'(x) - m psi_l(x) psi_l'(mx)] / [psi_l(mx) xi_l'(x) - m xi_l(x) psi_l'(mx)]
    with psi_l(z) = z j_l(z), xi_l(z) = z h_l(z)."""
    a = np.zeros(lmax, dtype=complex)
    b = np.zeros(lmax, dtype=complex)
    mx = m_rel * x
    for l in range(1, lmax + 1):
        psi_x = x * sf.sph_j(l, x)
        dpsi_x = x * sf.sph_j(l - 1, x) - l * sf.sph_j(l, x)
        psi_mx = mx * sf.sph_j(l, mx)
        dpsi_mx = mx * sf.sph_j(l - 1, mx) - l * sf.sph_j(l, mx)
        xi_x = x * sf.sph_h1(l, x)
        dxi_x = x * sf.sph_h1(l - 1, x) - l * sf.sph_h1(l, x)
        a[l - 1] = (m_rel * psi_mx * dpsi_x - psi_x * dpsi_mx) / (m_rel * psi_mx * dxi_x - xi_x * dpsi_mx)
        b[l - 1] = (psi_mx * dpsi_x - m_rel * psi_x * dpsi_mx) / (psi_mx * dxi_x - m_rel * xi_x * dpsi_mx)
    return a, b
