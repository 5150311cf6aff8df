"""Pins for the oracle's translation operator and coupling matrix (App. A.2,
Sec. 2.2).  CPU only.

The main pin is the SVWF addition theorem evaluated directly: outgoing waves
Psi^(3)_n(r + d) computed from their definition (App. A.1) must equal
sum_n' A_nn'(d) Psi^(1)_n'(r) for |r| < |d|.  Any error in a5/b5, in the
Legendre normalisation reading or in the phase conventions breaks it.
"""

import numpy as np
import pytest

from oracle import svwf, translation

K = 2 * np.pi / 550.0


@pytest.mark.parametrize("d,L", [((150.0, -80.0, 220.0), 2), ((-90.0, 40.0, -160.0), 3),
                                 ((0.0, 0.0, 260.0), 2), ((210.0, 0.0, 0.0), 2),
                                 ((120.0, 170.0, -90.0), 4), ((-60.0, -140.0, 250.0), 5),
                                 ((0.0, 0.0, -300.0), 4), ((-190.0, 75.0, 0.0), 5)])
def test_addition_theorem_direct(d, L):
    rng = np.random.default_rng(11)
    d = np.asarray(d)
    Lp = L + 18
    A = translation.translation_blocks(L, Lp, K, d[None, :])[0]
    u = rng.normal(size=(4, 3))
    # sample radius: the regular-wave series truncated at L' converges like
    # (|r| / |d|)^L', and the outgoing waves of degree 4-5 need the smaller
    # ratio to reach 1e-12 at L' = L + 18
    frac = 0.25 if L <= 3 else 0.15
    rpts = u / np.linalg.norm(u, axis=1)[:, None] * (frac * np.linalg.norm(d))
    idx_out = svwf.multi_indices(L)
    idx_in = svwf.multi_indices(Lp)
    basis = [svwf.svwf(1, tp, lp, mp, K, rpts) for (tp, lp, mp) in idx_in]
    for n, (tau, l, m) in enumerate(idx_out):
        lhs = svwf.svwf(3, tau, l, m, K, rpts + d[None, :])
        rhs = sum(A[n, q] * basis[q] for q in range(len(idx_in)))
        assert np.max(np.abs(lhs - rhs)) < 1e-9 * np.max(np.abs(lhs)), (tau, l, m)


def test_ab5_structure():
    # a5 real, b5 purely imaginary (the power of i is even for a5, odd for b5)
    for l in range(1, 5):
        for lp in range(1, 5):
            for m in range(-l, l + 1):
                for mp in range(-lp, lp + 1):
                    for p in range(abs(l - lp), l + lp + 1):
                        a5, b5 = translation.ab5(l, m, lp, mp, p)
                        assert abs(a5.imag) < 1e-15 and abs(b5.real) < 1e-15


def _term_count(L):
    na = nb = 0
    for l in range(1, L + 1):
        for lp in range(1, L + 1):
            for m in range(-l, l + 1):
                for mp in range(-lp, lp + 1):
                    for p in range(abs(l - lp), l + lp + 1):
                        if p < abs(m - mp):
                            continue
                        a5, b5 = translation.ab5(l, m, lp, mp, p)
                        na += a5 != 0
                        nb += b5 != 0
    return na, nb


def test_nonzero_term_counts():
    # counted nonzero (a5, b5) terms with p >= |m - m'|
    assert _term_count(2) == (109, 62)
    assert _term_count(3) == (461, 292)


def test_inversion_parity():
    # Psi_1lm(-r) = (-1)^l Psi_1lm(r), Psi_2lm(-r) = (-1)^{l+1} Psi_2lm(r) give
    # A_nn'(-d) = pi_n pi_n' A_nn'(d) with pi_n = (-1)^{l + [tau = 2]}
    L = 3
    d = np.array([[130.0, 75.0, -190.0]])
    A = translation.translation_blocks(L, L, K, d)[0]
    Am = translation.translation_blocks(L, L, K, -d)[0]
    par = np.array([(-1) ** (l + (t == 2)) for (t, l, m) in svwf.multi_indices(L)])
    assert np.max(np.abs(Am - par[:, None] * par[None, :] * A)) < 1e-13 * np.max(np.abs(A))
    # and the SVWF parities themselves
    r = np.array([[40.0, -25.0, 60.0]])
    for (t, l, m) in svwf.multi_indices(L):
        for nu in (1, 3):
            s = (-1) ** (l + (t == 2))
            assert np.allclose(svwf.svwf(nu, t, l, m, K, -r), s * svwf.svwf(nu, t, l, m, K, r), rtol=1e-12)


def test_reciprocity_transpose_with_m_reversed():
    # A_{n'n}(-d) = A_{~n ~n'}(d), ~n = (tau, l, -m)   =>  W^{ji}_{nn'} = W^{ij}_{~n' ~n}
    L = 3
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.normal(size=(1, 3)) * 200.0
        A = translation.translation_blocks(L, L, K, d)[0]
        Am = translation.translation_blocks(L, L, K, -d)[0]
        idx = svwf.multi_indices(L)
        flip = np.array([svwf.single_index(t, l, -m, L) for (t, l, m) in idx])
        assert np.max(np.abs(Am.T - A[np.ix_(flip, flip)])) < 1e-13 * np.max(np.abs(A))


def test_coupling_matrix_blocks_and_on_the_fly_rows():
    rng = np.random.default_rng(4)
    L = 2
    pos = rng.uniform(0, 800.0, size=(5, 3))
    W = translation.coupling_matrix(pos, K, L)
    nm = svwf.nmax_of(L)
    # block (i, i') is A(r_i - r_i') transposed, zero on the diagonal
    A01 = translation.translation_blocks(L, L, K, (pos[0] - pos[1])[None, :])[0]
    assert np.allclose(W[0:nm, nm:2 * nm], A01.T, rtol=1e-14, atol=0)
    assert np.all(W[0:nm, 0:nm] == 0)
    x = rng.normal(size=(5, nm)) + 1j * rng.normal(size=(5, nm))
    y = (W @ x.reshape(-1)).reshape(5, nm)
    rows = [0, 3, 4]
    yr = translation.coupling_matvec_rows(pos, K, L, x, rows)
    assert np.allclose(yr, y[rows], rtol=1e-13, atol=1e-13 * np.abs(y).max())


def test_blocks_are_continuous_at_the_poles():
    """As the translation vector approaches the z axis (where phi is
    undefined) the blocks converge to the on-axis block, at first order in the
    offset: sin(theta) enters as rho / |d| and no cos -> sin cancellation."""
    k = 2.0 * np.pi / 550.0
    for zsign in (1.0, -1.0):
        axis = translation.coupling_blocks(3, k, np.array([[0.0, 0.0, zsign * 400.0]]), np.zeros((1, 3)))[0]
        scale = np.abs(axis).max()
        errs = []
        for eps in (1e-2, 1e-4, 1e-6):
            for phi in (0.0, 1.0, 2.5):
                d = np.array([[eps * np.cos(phi), eps * np.sin(phi), zsign * 400.0]])
                W = translation.coupling_blocks(3, k, d, np.zeros((1, 3)))[0]
                errs.append(np.abs(W - axis).max() / scale)
        # offsets two decades apart: the deviation falls by the same factor
        # (first order, no precision floor down to 1e-6 nm)
        e = np.array(errs).reshape(3, 3).max(axis=1)
        assert e[0] < 1e-4
        assert abs(e[1] / e[0] - 1e-2) < 1e-4 and abs(e[2] / e[1] - 1e-2) < 1e-4
