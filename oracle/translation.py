"""SVWF translation operator and coupling matrix (Sec. 2.2, App. A.2), FP64.

Test infrastructure only (see the package docstring).

Addition theorem (App. A.2):  Psi^(3)_n(r + d) = sum_n' A_{nn'}(d) Psi^(1)_n'(r)
for |r| < |d|, with

  A_{tau l m, tau' l' m'}(d) = delta_{tau tau'} A_{ml,m'l'}(d)
                               + (1 - delta_{tau tau'}) B_{ml,m'l'}(d)
  A_{ml,m'l'}(d) = e^{i(m-m')phi_d} sum_{p=|l-l'|}^{l+l'}   a5(l,m|l',m'|p) h_p(kd) P_p^{|m-m'|}(cos theta_d)
  B_{ml,m'l'}(d) = e^{i(m-m')phi_d} sum_{p=|l-l'|+1}^{l+l'} b5(l,m|l',m'|p) h_p(kd) P_p^{|m-m'|}(cos theta_d)

(the paper overloads "p" for polarisation and for the sum index; here the
polarisation is tau and p is only the sum index).  The coupling matrix is the
transpose of A from r_i' to r_i (Sec. 2.2):  W^{ii'}_{nn'} = A_{n'n}(r_i - r_i').
"""

from functools import lru_cache

import numpy as np

from . import special as sf
from .svwf import multi_indices, nmax_of


@lru_cache(maxsize=None)
def ab5(l, m, lp, mp, p):
    """(a5, b5)(l,m|l',m'|p) exactly as printed in App. A.2 (complex values)."""
    ipow = abs(m - mp) - abs(m) - abs(mp) + lp - l + p
    phase = (1j) ** (ipow % 4) * (-1) ** ((m - mp) % 2)
    fac1 = np.sqrt((2 * l + 1) * (2 * lp + 1) / (2.0 * l * (l + 1) * lp * (lp + 1)))
    w_m = sf.wigner3j(l, lp, p, m, -mp, mp - m)
    a5 = 0.0
    b5 = 0.0
    if w_m != 0.0:
        w0 = sf.wigner3j(l, lp, p, 0, 0, 0)
        a5 = phase * (l * (l + 1) + lp * (lp + 1) - p * (p + 1)) * np.sqrt(2 * p + 1) * fac1 * w_m * w0
        if p >= 1:
            prod = (l + lp + 1 + p) * (l + lp + 1 - p) * (p + l - lp) * (p - l + lp) * (2 * p + 1)
            w1 = sf.wigner3j(l, lp, p - 1, 0, 0, 0)
            if prod > 0 and w1 != 0.0:
                b5 = phase * np.sqrt(prod) * fac1 * w_m * w1
    return complex(a5), complex(b5)


def _pair_geometry(d):
    d = np.atleast_2d(np.asarray(d, dtype=float))
    dist = np.sqrt(np.sum(d * d, axis=1))
    rho = np.hypot(d[:, 0], d[:, 1])
    ct = d[:, 2] / dist
    st = rho / dist
    phi = np.arctan2(d[:, 1], d[:, 0])
    return dist, ct, st, phi


def translation_blocks(lmax_out, lmax_in, k, d):
    """A_{nn'}(d) for many translation vectors d.

    Returns complex array (npairs, nmax(lmax_out), nmax(lmax_in)); row index n
    (the translated outgoing wave) runs over lmax_out, column index n' (the
    regular wave) over lmax_in.
    """
    dist, ct, st, phi = _pair_geometry(d)
    npairs = dist.shape[0]
    pmax = lmax_out + lmax_in
    h = [sf.sph_h1(p, k * dist) for p in range(pmax + 1)]
    P = {}
    for p in range(pmax + 1):
        for mu in range(p + 1):
            P[(p, mu)] = sf.legendre_p(p, mu, ct, st)
    idx_out = multi_indices(lmax_out)
    idx_in = multi_indices(lmax_in)
    nh_out = lmax_out * (lmax_out + 2)
    nh_in = lmax_in * (lmax_in + 2)
    A = np.zeros((npairs, 2 * nh_out, 2 * nh_in), dtype=complex)
    for a, (tau, l, m) in enumerate(idx_out[:nh_out]):
        for b, (taup, lp, mp) in enumerate(idx_in[:nh_in]):
            mu = abs(m - mp)
            eph = np.exp(1j * (m - mp) * phi)
            sa = np.zeros(npairs, dtype=complex)
            sb = np.zeros(npairs, dtype=complex)
            for p in range(abs(l - lp), l + lp + 1):
                if p < mu:
                    continue
                a5, b5 = ab5(l, m, lp, mp, p)
                term = h[p] * P[(p, mu)]
                if a5 != 0:
                    sa += a5 * term
                if b5 != 0 and p >= abs(l - lp) + 1:
                    sb += b5 * term
            Ablk = eph * sa
            Bblk = eph * sb
            A[:, a, b] = Ablk
            A[:, a + nh_out, b + nh_in] = Ablk
            A[:, a, b + nh_in] = Bblk
            A[:, a + nh_out, b] = Bblk
    return A


def coupling_blocks(lmax, k, r_recv, r_src):
    """W^{ii'} blocks for receivers r_recv[q] and sources r_src[q]:
    W^{ii'}_{nn'} = A_{n'n}(r_i - r_i'), shape (npairs, nmax, nmax)."""
    d = np.asarray(r_recv, dtype=float) - np.asarray(r_src, dtype=float)
    A = translation_blocks(lmax, lmax, k, d)
    return np.transpose(A, (0, 2, 1))


def coupling_matrix(positions, k, lmax):
    """Dense coupling matrix W, shape (N*nmax, N*nmax), zero diagonal blocks."""
    pos = np.asarray(positions, dtype=float)
    N = pos.shape[0]
    nm = nmax_of(lmax)
    W = np.zeros((N * nm, N * nm), dtype=complex)
    ii, jj = np.nonzero(~np.eye(N, dtype=bool))
    if ii.size:
        blocks = coupling_blocks(lmax, k, pos[ii], pos[jj])
        for q in range(ii.size):
            i, j = ii[q], jj[q]
            W[i * nm:(i + 1) * nm, j * nm:(j + 1) * nm] = blocks[q]
    return W


def coupling_matvec_rows(positions, k, lmax, x, rows, chunk=4096):
    """y_i = sum_{j != i} W^{ij} x_j for the receivers listed in ``rows``.

    ``x`` has shape (N, nmax) (or (nrhs, N, nmax)); returns (len(rows), nmax)
    (or (nrhs, len(rows), nmax)).  Blocks are built on the fly, no dense W.
    """
    pos = np.asarray(positions, dtype=float)
    N = pos.shape[0]
    nm = nmax_of(lmax)
    xx = np.asarray(x)
    single = xx.ndim == 2
    if single:
        xx = xx[None]
    out = np.zeros((xx.shape[0], len(rows), nm), dtype=complex)
    for a, i in enumerate(rows):
        src = np.array([j for j in range(N) if j != i], dtype=int)
        for c0 in range(0, src.size, chunk):
            js = src[c0:c0 + chunk]
            blk = coupling_blocks(lmax, k, np.repeat(pos[i][None, :], js.size, axis=0), pos[js])
            out[:, a, :] += np.einsum("qab,rqb->ra", blk, xx[:, js, :])
    return out[0] if single else out
