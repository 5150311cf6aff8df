"""Master equation, dense solve, GMRES and cross sections (Sec. 2.2), FP64.

Test infrastructure only (see the package docstring).

Multiple-scattering equations (Sec. 2.2):
  a^i = a_in^i + sum_{i' != i} W^{ii'} b^{i'},     b^i = T^i a^i
Eliminating a gives the master equation  sum M^{ii'} b^{i'} = T^i a_in^i  with
  M^{ii'}_{nn'} = delta_{nn'} delta_{ii'} - sum_n'' T^i_{nn''} W^{ii'}_{n''n'}.
Because T is diagonal, (M x)_i = x_i - T^i (W x)_i.

The oracle's solution is the plain definition: assemble the dense M and solve
it with LAPACK's LU (scipy.linalg.solve).  The iterative solver of Sec. 3.2
(GMRES) reaches the same vector up to its tolerance.
"""

import numpy as np
import scipy.linalg as sla

from .translation import coupling_matrix


def master_matrix(tdiag, W):
    """M = I - diag(T) W  (tdiag flattened to length N*nmax)."""
    t = np.asarray(tdiag).reshape(-1)
    return np.eye(t.size, dtype=complex) - t[:, None] * W


def solve_dense(positions, k, lmax, tdiag, a_in):
    """b solving M b = T a_in by dense LU.  ``a_in``: (N, nmax) or (nrhs, N, nmax)."""
    W = coupling_matrix(positions, k, lmax)
    M = master_matrix(tdiag, W)
    a = np.asarray(a_in)
    single = a.ndim == 2
    if single:
        a = a[None]
    t = np.asarray(tdiag).reshape(-1)
    rhs = (t[None, :] * a.reshape(a.shape[0], -1)).T
    b = sla.solve(M, rhs)
    b = b.T.reshape(a.shape)
    return b[0] if single else b


def apply_M(W, tdiag, x):
    """M x = x - T (W x) with a dense W; x shaped (N, nmax)."""
    xf = np.asarray(x).reshape(-1)
    t = np.asarray(tdiag).reshape(-1)
    return (xf - t * (W @ xf)).reshape(np.shape(x))


def _givens(a, b):
    """Complex Givens rotation [c s; -conj(s) c] (c real) mapping (a, b) -> (r, 0)."""
    if b == 0:
        return 1.0, 0.0
    if a == 0:
        return 0.0, 1.0
    den = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    return abs(a) / den, (a / abs(a)) * np.conj(b) / den


def gmres(matvec, rhs, x0=None, tol=1e-10, restart=100, maxiter=1000, precond=None):
    """Restarted GMRES with right preconditioning (textbook form, Barrett et al.):
    solves A x = rhs, stopping when ||rhs - A x|| <= tol ||rhs||.

    ``matvec``/``precond`` act on flat complex vectors.  Modified Gram-Schmidt,
    Givens rotations.  Returns (x, relative residual history, iterations).
    """
    rhs = np.asarray(rhs, dtype=complex).reshape(-1)
    n = rhs.size
    x = np.zeros(n, dtype=complex) if x0 is None else np.asarray(x0, dtype=complex).reshape(-1).copy()
    Pinv = (lambda v: v) if precond is None else precond
    bnorm = np.linalg.norm(rhs)
    if bnorm == 0:
        return np.zeros(n, dtype=complex), [0.0], 0
    hist = []
    its = 0
    while True:
        r = rhs - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm or its >= maxiter:
            break
        m = min(restart, maxiter - its)
        V = np.zeros((m + 1, n), dtype=complex)
        H = np.zeros((m + 1, m), dtype=complex)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=complex)
        g = np.zeros(m + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        kk = 0
        while kk < m:
            w = matvec(Pinv(V[kk]))
            for j in range(kk + 1):
                H[j, kk] = np.vdot(V[j], w)
                w = w - H[j, kk] * V[j]
            H[kk + 1, kk] = np.linalg.norm(w)
            if H[kk + 1, kk] != 0:
                V[kk + 1] = w / H[kk + 1, kk]
            for j in range(kk):
                t = cs[j] * H[j, kk] + sn[j] * H[j + 1, kk]
                H[j + 1, kk] = -np.conj(sn[j]) * H[j, kk] + cs[j] * H[j + 1, kk]
                H[j, kk] = t
            cs[kk], sn[kk] = _givens(H[kk, kk], H[kk + 1, kk])
            H[kk, kk] = cs[kk] * H[kk, kk] + sn[kk] * H[kk + 1, kk]
            H[kk + 1, kk] = 0.0
            g[kk + 1] = -np.conj(sn[kk]) * g[kk]
            g[kk] = cs[kk] * g[kk]
            kk += 1
            its += 1
            if abs(g[kk]) <= tol * bnorm:
                break
        y = sla.solve_triangular(H[:kk, :kk], g[:kk])
        x = x + Pinv(V[:kk].T @ y)
    return x, hist, its


# ----------------------------------------------------------------------------
# cross sections (normalisation fixed by the single-sphere Mie pin)
# ----------------------------------------------------------------------------
#
# With the SVWF normalisation of App. A.1 the outgoing wave sum_n b_n Psi^(3)_n
# carries power proportional to (pi/k^2) sum |b_n|^2, and for one sphere in a
# plane wave of unit amplitude these give the Mie series
#   C_ext = -(pi/k^2) Re sum a_n^* b_n ,   C_sca = (pi/k^2) sum |b_n|^2 .

def c_ext(k, a_in, b, E0=1.0):
    """Extinction cross section  -(pi/k^2) Re sum_i sum_n conj(a_in) b / |E0|^2."""
    return float(-np.pi / k ** 2 * np.real(np.vdot(np.asarray(a_in).reshape(-1), np.asarray(b).reshape(-1)))
                 / abs(E0) ** 2)


def c_abs(k, tdiag, b, E0=1.0):
    """Absorption cross section -(pi/k^2) sum |b_n|^2 (Re(1/Q_n) + 1) / |E0|^2
    (b = T a for each sphere's total exciting field a)."""
    t = np.asarray(tdiag).reshape(-1)
    bb = np.asarray(b).reshape(-1)
    return float(-np.pi / k ** 2 * np.sum(np.abs(bb) ** 2 * (np.real(1.0 / t) + 1.0)) / abs(E0) ** 2)


def c_sca_single(k, b, E0=1.0):
    """Scattering cross section of ONE sphere's expansion: (pi/k^2) sum |b_n|^2."""
    return float(np.pi / k ** 2 * np.sum(np.abs(np.asarray(b)) ** 2) / abs(E0) ** 2)
