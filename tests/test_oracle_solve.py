"""Pins for the oracle's master-equation solve, far field and cross sections
(Sec. 2.2, App. D).  CPU only."""

import numpy as np
import pytest

import synth
from oracle import farfield, incident, mie, precond, solve, svwf, translation

K = 2 * np.pi / 550.0


def _cluster(N, L, n=1.52 + 0j, seed=0, radius=100.0, fill=0.2):
    sc = synth.random_cluster(90, seed, N, L, radius=radius, fill=fill, n=n)
    t = mie.t_diagonal(L, sc.k, sc.radii, sc.n_rel)
    a = incident.plane_wave_coeffs(L, sc.k, sc.positions, 0.3, 0.8, 2)
    return sc, t, a


def test_single_sphere_solution_is_T_a():
    sc, t, a = _cluster(1, 3)
    b = solve.solve_dense(sc.positions, sc.k, 3, t, a)
    assert np.allclose(b, t * a, rtol=1e-14, atol=0)


def test_dense_solution_satisfies_the_multiple_scattering_equations():
    # a^i = a_in^i + sum_{i'} W^{ii'} b^{i'} and b^i = T^i a^i  (Sec. 2.2)
    sc, t, a = _cluster(6, 3, n=1.5 + 0.02j)
    b = solve.solve_dense(sc.positions, sc.k, 3, t, a)
    W = translation.coupling_matrix(sc.positions, sc.k, 3)
    a_tot = a.reshape(-1) + W @ b.reshape(-1)
    assert np.allclose(b.reshape(-1), t.reshape(-1) * a_tot, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n", [1.52 + 0j, 1.5 + 0.05j])
def test_optical_theorem(n):
    # C_ext (forward/interference form) = C_sca (quadrature of |g|^2 over all
    # directions) + C_abs (per-sphere), and C_abs = 0 for real n
    L = 3
    sc, t, a = _cluster(4, L, n=n, seed=1)
    b = solve.solve_dense(sc.positions, sc.k, L, t, a)
    ce = solve.c_ext(sc.k, a, b)
    ca = solve.c_abs(sc.k, t, b)
    cs = farfield.c_sca_quadrature(L, sc.k, sc.positions, b, n_beta=48, n_alpha=96)
    assert abs(ce - (cs + ca)) < 1e-9 * ce
    if np.imag(n) == 0:
        assert abs(ca) < 1e-12 * ce
    else:
        assert ca > 0.01 * ce


def test_extinction_equals_forward_amplitude():
    # C_ext = -(8 pi^2 / k^2) Re[e^* . g(k_in)] for the incident polarisation
    L = 3
    sc, t, a = _cluster(3, L, seed=2)
    beta, alpha, pol = 0.3, 0.8, 2
    b = solve.solve_dense(sc.positions, sc.k, L, t, a)
    g = farfield.farfield_amplitude(L, sc.k, sc.positions, b, [[beta, alpha]])[0]
    assert abs(solve.c_ext(sc.k, a, b) - (-8 * np.pi ** 2 / sc.k ** 2 * np.real(g[pol - 1]))) < 1e-10 * solve.c_ext(sc.k, a, b)


def test_far_field_matches_direct_large_r_evaluation():
    # E_scat(r) ~ -2 pi i e^{ikr}/(kr) sum_j g_j e_j  for kr -> infinity
    L = 3
    sc, t, a = _cluster(3, L, seed=3)
    b = solve.solve_dense(sc.positions, sc.k, L, t, a)
    R = 4e9   # corrections are O(k d^2 / R) with d the cluster size
    for beta, alpha in [(0.4, 0.2), (2.1, -1.3), (1.2, 2.5)]:
        u = np.array([np.sin(beta) * np.cos(alpha), np.sin(beta) * np.sin(alpha), np.cos(beta)])
        r = (R * u)[None, :]
        E = np.zeros(3, dtype=complex)
        for i in range(sc.N):
            E += svwf.field_expansion(3, b[i], L, sc.k, r, origin=sc.positions[i])[0]
        g = farfield.farfield_amplitude(L, sc.k, sc.positions, b, [[beta, alpha]])[0]
        e_a, e_b = svwf.pvwf_unit_vectors(alpha, beta)
        Ef = -2j * np.pi * np.exp(1j * sc.k * R) / (sc.k * R) * (g[0] * e_a + g[1] * e_b)
        assert np.linalg.norm(E - Ef) < 2e-6 * np.linalg.norm(Ef)


def test_lmax_convergence_two_spheres():
    # the change of C_ext from L to L+1 falls off geometrically
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 150.0, 170.0]])
    radii = np.array([100.0, 100.0])
    ce = []
    for L in range(1, 10):
        t = mie.t_diagonal(L, K, radii, [1.52, 1.52])
        a = incident.plane_wave_coeffs(L, K, pos, 0.0, 0.0, 2)
        b = solve.solve_dense(pos, K, L, t, a)
        ce.append(solve.c_ext(K, a, b))
    diffs = np.abs(np.diff(ce))
    # nearly touching spheres (gap 27 nm): ratio ~ 0.25 once L >= 3
    assert np.all(diffs[3:] < 0.4 * diffs[2:-1])
    assert diffs[-1] < 1e-6 * ce[-1]


def test_distant_spheres_decouple():
    # |r_1 - r_2| -> infinity: W -> 0 like 1/(kd) and b -> T a_in
    L = 3
    pos = np.array([[0.0, 0.0, 0.0], [3e7, 1e7, -2e7]])
    t = mie.t_diagonal(L, K, [100.0, 120.0], [1.52, 1.6])
    a = incident.plane_wave_coeffs(L, K, pos, 0.2, 0.1, 1)
    b = solve.solve_dense(pos, K, L, t, a)
    assert np.max(np.abs(b - t * a)) < 1e-4 * np.max(np.abs(t * a))


def test_gmres_matches_dense_lu():
    L = 2
    sc, t, a = _cluster(3, L, n=1.6 + 0.01j, seed=4, fill=0.3)
    b = solve.solve_dense(sc.positions, sc.k, L, t, a)
    W = translation.coupling_matrix(sc.positions, sc.k, L)
    M = solve.master_matrix(t, W)
    x, hist, its = solve.gmres(lambda v: M @ v, (t * a).reshape(-1), tol=1e-13, restart=7)
    assert hist[-1] <= 1e-13
    assert np.linalg.norm(x - b.reshape(-1)) < 1e-11 * np.linalg.norm(b)


def test_block_preconditioner():
    L = 2
    sc, t, a = _cluster(12, L, seed=5, fill=0.25)
    W = translation.coupling_matrix(sc.positions, sc.k, L)
    M = solve.master_matrix(t, W)
    perm, off = precond.partition(sc.positions, 250.0)
    # every sphere once; contiguous blocks share one cuboid
    assert sorted(perm.tolist()) == list(range(sc.N))
    lo = sc.positions.min(axis=0)
    cell = np.floor((sc.positions - lo) / 250.0).astype(int)
    for q in range(len(off) - 1):
        ids = perm[off[q]:off[q + 1]]
        assert len({tuple(c) for c in cell[ids]}) == 1
    keys = [tuple(cell[perm[off[q]]][::-1]) for q in range(len(off) - 1)]
    assert keys == sorted(keys)
    P = precond.BlockPreconditioner(sc.positions, sc.k, L, t, 250.0)
    y = synth.random_vector(90, 1, (sc.N, svwf.nmax_of(L)))
    x = P.apply(y)
    # each block of M times x reproduces y on that block
    nm = svwf.nmax_of(L)
    for ids, _ in P.blocks:
        sel = np.concatenate([np.arange(i * nm, (i + 1) * nm) for i in ids])
        assert np.allclose(M[np.ix_(sel, sel)] @ x.reshape(-1)[sel], y.reshape(-1)[sel], rtol=1e-11, atol=1e-11)
    # one block covering everything is the exact inverse: GMRES converges at once
    Pall = precond.BlockPreconditioner(sc.positions, sc.k, L, t, 1e9)
    xs, hist, its = solve.gmres(lambda v: M @ v, (t * a).reshape(-1), tol=1e-12,
                                precond=lambda v: Pall.apply(v.reshape(sc.N, nm)).reshape(-1))
    assert its <= 2
