"""Spherical and plane vector wave functions (App. A.1), FP64, Cartesian output.

Test infrastructure only (see the package docstring).

Psi^(nu)_{tau l m}(r) for nu = 1 (regular, z_l = j_l) and nu = 3 (outgoing,
z_l = h_l^(1)), written out from the explicit form in App. A.1:

  Psi_1lm = e^{i m phi}/sqrt(2l(l+1)) z_l(kr) ( i m pi_l^|m| e_theta - tau_l^|m| e_phi )
  Psi_2lm = e^{i m phi}/sqrt(2l(l+1)) ( l(l+1) z_l(kr)/(kr) P_l^|m| e_r
            + [d_{kr}(kr z_l(kr))]/(kr) ( tau_l^|m| e_theta + i m pi_l^|m| e_phi ) )

Phi_1(alpha,beta;r) = e^{i k.r} e_alpha, Phi_2 = e^{i k.r} e_beta, with
(k, beta, alpha) the spherical coordinates of the wave vector (App. A.1).
"""

import numpy as np

from . import special as sf


def _spherical_coords(r):
    r = np.atleast_2d(np.asarray(r, dtype=float))
    x, y, z = r[:, 0], r[:, 1], r[:, 2]
    rho = np.hypot(x, y)
    rr = np.sqrt(x * x + y * y + z * z)
    ct = np.where(rr > 0, z / np.where(rr > 0, rr, 1.0), 1.0)
    st = np.where(rr > 0, rho / np.where(rr > 0, rr, 1.0), 0.0)
    phi = np.arctan2(y, x)
    return rr, ct, st, phi


def _unit_vectors(ct, st, phi):
    cp, sp = np.cos(phi), np.sin(phi)
    e_r = np.stack([st * cp, st * sp, ct], axis=-1)
    e_t = np.stack([ct * cp, ct * sp, -st], axis=-1)
    e_p = np.stack([-sp, cp, np.zeros_like(cp)], axis=-1)
    return e_r, e_t, e_p


def svwf(nu, tau, l, m, k, r):
    """Psi^(nu)_{tau l m}(r), returned as complex array (npts, 3) in Cartesian
    components.  ``k`` is the (real) wavenumber of the medium."""
    rr, ct, st, phi = _spherical_coords(r)
    e_r, e_t, e_p = _unit_vectors(ct, st, phi)
    kr = k * rr
    if nu == 1:
        z = sf.sph_j(l, kr)
        dz = sf.dxxj(l, kr)
        # limits kr -> 0 of z_l/kr and d(kr z_l)/kr (nonzero only for l = 1)
        with np.errstate(divide="ignore", invalid="ignore"):
            z_kr = np.where(kr > 0, z / np.where(kr > 0, kr, 1.0), (1.0 / 3.0) if l == 1 else 0.0)
            dz_kr = np.where(kr > 0, dz / np.where(kr > 0, kr, 1.0), (2.0 / 3.0) if l == 1 else 0.0)
    elif nu == 3:
        z = sf.sph_h1(l, kr)
        dz = sf.dxxh(l, kr)
        z_kr = z / kr
        dz_kr = dz / kr
    else:
        raise ValueError("nu must be 1 or 3")
    am = abs(m)
    P = sf.legendre_p(l, am, ct, st)
    pi = sf.legendre_pi(l, am, ct, st)
    ta = sf.legendre_tau(l, am, ct, st)
    pref = np.exp(1j * m * phi) / np.sqrt(2.0 * l * (l + 1))
    if tau == 1:
        vec = (z[:, None] * ((1j * m * pi)[:, None] * e_t - ta[:, None] * e_p))
    elif tau == 2:
        vec = ((l * (l + 1) * z_kr * P)[:, None] * e_r
               + dz_kr[:, None] * (ta[:, None] * e_t + (1j * m * pi)[:, None] * e_p))
    else:
        raise ValueError("tau must be 1 or 2")
    return pref[:, None] * vec


def pvwf_unit_vectors(alpha, beta):
    """Unit vectors e_alpha, e_beta of the plane-wave direction (beta, alpha)."""
    ca, sa, cb, sb = np.cos(alpha), np.sin(alpha), np.cos(beta), np.sin(beta)
    e_a = np.array([-sa, ca, 0.0])
    e_b = np.array([cb * ca, cb * sa, -sb])
    return e_a, e_b


def pvwf(j, alpha, beta, k, r):
    """Phi_j(alpha, beta; r) (App. A.1) as complex array (npts, 3)."""
    r = np.atleast_2d(np.asarray(r, dtype=float))
    kvec = k * np.array([np.sin(beta) * np.cos(alpha), np.sin(beta) * np.sin(alpha), np.cos(beta)])
    e_a, e_b = pvwf_unit_vectors(alpha, beta)
    ph = np.exp(1j * r @ kvec)
    e = e_a if j == 1 else e_b
    return ph[:, None] * e[None, :]


def single_index(tau, l, m, lmax):
    """n = (tau-1) L(L+2) + l(l+1) - 1 + m (0-based)."""
    return (tau - 1) * lmax * (lmax + 2) + l * (l + 1) - 1 + m


def multi_indices(lmax):
    """List of (tau, l, m) in coefficient order."""
    out = []
    for tau in (1, 2):
        for l in range(1, lmax + 1):
            for m in range(-l, l + 1):
                out.append((tau, l, m))
    return out


def nmax_of(lmax):
    return 2 * lmax * (lmax + 2)


def field_expansion(nu, coeffs, lmax, k, r, origin=(0.0, 0.0, 0.0)):
    """sum_n c_n Psi^(nu)_n(r - origin), complex array (npts, 3)."""
    r = np.atleast_2d(np.asarray(r, dtype=float)) - np.asarray(origin, dtype=float)[None, :]
    out = np.zeros((r.shape[0], 3), dtype=complex)
    for n, (tau, l, m) in enumerate(multi_indices(lmax)):
        if coeffs[n] != 0:
            out += coeffs[n] * svwf(nu, tau, l, m, k, r)
    return out
