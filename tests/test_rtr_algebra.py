"""The algebra behind the coupling kernel's rotation-translation-rotation
form (Sec. 5), checked on the CPU against the oracle's dense coupling blocks
(App. A.2).  The Wigner small-d matrices are written out here from Wigner's
explicit formula, independently of the kernel's tables.

* W(d) = D^H W_z(k|d|) D, with D = blockdiag_l R^l(theta) diag(e^{i m phi})
  and R^l_{mu m} = s_mu s_m d^l_{m mu}(theta), s_m = (-1)^m for m >= 0, else 1;
* W_z (translation along +z) couples equal m only;
* per tau block W = [[A, B], [B, A]], so x+- = x_1 +- x_2 decouple;
* mirror: A(l, l', -mu) = A(l, l', mu), B(l, l', -mu) = -B(l, l', mu);
* transpose: entry (l', l) = (-1)^{l + l'} entry (l, l') of A and B alike;
* rotation rows: R_{-mu,-m} = R_{mu m} and R_{-mu,m} = R_{mu,-m}.
"""

from math import factorial

import numpy as np
import pytest

from oracle import svwf, translation

L = 4
K = 2.0 * np.pi / 550.0


def wigner_small_d(l, mp, m, beta):
    """d^l_{m' m}(beta) by Wigner's explicit sum."""
    s = 0.0
    for k in range(0, 2 * l + 1):
        a1, a2, a3 = l + m - k, l - k - mp, k - m + mp
        if a1 < 0 or a2 < 0 or a3 < 0:
            continue
        num = np.sqrt(factorial(l + mp) * factorial(l - mp) * factorial(l + m) * factorial(l - m))
        den = factorial(a1) * factorial(k) * factorial(a2) * factorial(a3)
        s += (-1) ** (k - m + mp) * num / den * np.cos(beta / 2) ** (2 * l - 2 * k + m - mp) \
            * np.sin(beta / 2) ** (2 * k - m + mp)
    return s


def sgn(m):
    return (-1) ** m if m >= 0 else 1


def rot(l, mu, m, theta):
    return sgn(mu) * sgn(m) * wigner_small_d(l, m, mu, theta)


def wz(dist):
    return translation.coupling_blocks(L, K, np.array([[0.0, 0.0, dist]]), np.zeros((1, 3)))[0]


def rotation_matrix(theta, phi):
    idx = svwf.multi_indices(L)
    D = np.zeros((len(idx), len(idx)), dtype=complex)
    for a, (t, l, mu) in enumerate(idx):
        for b, (t2, l2, m) in enumerate(idx):
            if t == t2 and l == l2:
                D[a, b] = rot(l, mu, m, theta) * np.exp(1j * m * phi)
    return D


@pytest.mark.parametrize("d", [(180.0, -240.0, 330.0), (0.0, 0.0, -400.0), (1.0e-3, 0.0, 500.0),
                               (-700.0, 50.0, -20.0), (2500.0, 2600.0, 900.0)])
def test_rotation_translation_rotation_equals_dense_block(d):
    d = np.asarray(d)
    dist = np.linalg.norm(d)
    theta, phi = np.arctan2(np.hypot(d[0], d[1]), d[2]), np.arctan2(d[1], d[0])  # accurate at the poles
    W = translation.coupling_blocks(L, K, d[None, :], np.zeros((1, 3)))[0]
    D = rotation_matrix(theta, phi)
    W2 = D.conj().T @ wz(dist) @ D
    assert np.max(np.abs(W2 - W)) <= 1e-12 * np.max(np.abs(W))


def test_axial_block_structure():
    idx = svwf.multi_indices(L)
    nh = len(idx) // 2
    W = wz(430.0)
    scale = np.max(np.abs(W))
    for a, (t, l, mu) in enumerate(idx):
        for b, (t2, l2, m) in enumerate(idx):
            if mu != m:
                assert abs(W[a, b]) <= 1e-14 * scale
    A, B = W[:nh, :nh], W[:nh, nh:]
    # tau structure [[A, B], [B, A]]
    assert np.allclose(W[nh:, nh:], A, rtol=0, atol=1e-14 * scale)
    assert np.allclose(W[nh:, :nh], B, rtol=0, atol=1e-14 * scale)
    pos = {(l, m): q for q, (t, l, m) in enumerate(idx[:nh])}
    for l in range(1, L + 1):
        for lp in range(1, L + 1):
            for mu in range(0, min(l, lp) + 1):
                i, j = pos[(l, mu)], pos[(lp, mu)]
                im, jm = pos[(l, -mu)], pos[(lp, -mu)]
                # mirror mu -> -mu
                assert abs(A[im, jm] - A[i, j]) <= 1e-13 * scale
                assert abs(B[im, jm] + B[i, j]) <= 1e-13 * scale
                # transpose (l, l') -> (l', l)
                sign = (-1) ** (l + lp)
                assert abs(A[j, i] - sign * A[i, j]) <= 1e-13 * scale
                assert abs(B[j, i] - sign * B[i, j]) <= 1e-13 * scale


def test_plus_minus_basis_decouples():
    rng = np.random.default_rng(3)
    d = rng.normal(size=3) * 400.0
    W = translation.coupling_blocks(L, K, d[None, :], np.zeros((1, 3)))[0]
    nh = W.shape[0] // 2
    x1 = rng.normal(size=nh) + 1j * rng.normal(size=nh)
    x2 = rng.normal(size=nh) + 1j * rng.normal(size=nh)
    y = W @ np.concatenate([x1, x2])
    A, B = W[:nh, :nh], W[:nh, nh:]
    assert np.allclose(y[:nh] + y[nh:], (A + B) @ (x1 + x2), atol=1e-12 * np.abs(y).max())
    assert np.allclose(y[:nh] - y[nh:], (A - B) @ (x1 - x2), atol=1e-12 * np.abs(y).max())


@pytest.mark.parametrize("theta", [0.3, 1.2, 2.9])
def test_rotation_row_symmetry(theta):
    for l in range(1, 6):
        for mu in range(0, l + 1):
            for m in range(0, l + 1):
                assert abs(rot(l, -mu, -m, theta) - rot(l, mu, m, theta)) <= 1e-13
                assert abs(rot(l, -mu, m, theta) - rot(l, mu, -m, theta)) <= 1e-13
        # each R^l is orthogonal (a rotation of real-weighted harmonics)
        R = np.array([[rot(l, mu, m, theta) for m in range(-l, l + 1)] for mu in range(-l, l + 1)])
        assert np.allclose(R @ R.T, np.eye(2 * l + 1), atol=1e-13)
