"""Reflected / transmitted power (App. D) of the oracle, pinned by
  * the incident beam alone (b = 0): T = 1 and R = 0, which checks the
    closed-form incident power against the quadrature of |g_in|^2;
  * energy conservation for lossless spheres: R + T = 1 (the paper reports
    this balance to 1e-3 for its runs; with the exact dense solution of a
    small case and converged quadrature it holds to rounding, 1e-10);
  * absorbing spheres: R + T < 1."""

import numpy as np

import synth
from oracle import incident, mie, power, solve


def _gauss_case(n_sphere, seed=0, N=6, L=3):
    sc = synth.random_cluster(71, seed, N, L, radius=110.0, fill=0.12, n=n_sphere)
    w, focus, aG = 1200.0, (30.0, -20.0, 0.0), -np.pi / 2
    t = mie.t_diagonal(L, sc.k, sc.radii, sc.n_rel)
    a = incident.gaussian_beam_coeffs(L, sc.k, sc.positions, w, focus, aG, n_beta=256)
    b = solve.solve_dense(sc.positions, sc.k, L, t, a)
    return sc, b, w, focus, aG


def test_incident_beam_alone():
    sc, b, w, focus, aG = _gauss_case(1.5 + 0j)
    R, T = power.reflect_transmit(sc.lmax, sc.k, sc.positions, 0.0 * b, w, focus, aG, n_beta=96, n_alpha=32)
    assert abs(T - 1.0) < 1e-9 and R == 0.0


def test_energy_balance_lossless():
    sc, b, w, focus, aG = _gauss_case(1.6 + 0j)
    R, T = power.reflect_transmit(sc.lmax, sc.k, sc.positions, b, w, focus, aG, n_beta=96, n_alpha=96)
    assert R > 1e-4 and T < 1.0
    assert abs(R + T - 1.0) < 1e-10


def test_absorbing_spheres_lose_power():
    sc, b, w, focus, aG = _gauss_case(1.6 + 0.2j)
    R, T = power.reflect_transmit(sc.lmax, sc.k, sc.positions, b, w, focus, aG, n_beta=96, n_alpha=96)
    assert R + T < 1.0 - 1e-4
