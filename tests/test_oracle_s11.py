"""S11 of the oracle (far-field intensity averaged over azimuth and over TE
and TM incidence, Sec. 4) for one sphere equals, up to one constant, the
unpolarised Mie phase function (|S1|^2 + |S2|^2)/2 with S1, S2 from the
Bohren-Huffman amplitude functions (textbook recurrences for pi_n, tau_n)."""

import numpy as np

from oracle import farfield, incident, mie


def _bh_s1_s2(a, b, theta):
    mu = np.cos(theta)
    n_max = len(a)
    pi_prev, pi_cur = np.zeros_like(mu), np.ones_like(mu)  # pi_0, pi_1
    S1 = np.zeros_like(mu, dtype=complex)
    S2 = np.zeros_like(mu, dtype=complex)
    for n in range(1, n_max + 1):
        if n > 1:
            pi_next = ((2 * n - 1) / (n - 1)) * mu * pi_cur - (n / (n - 1)) * pi_prev
            pi_prev, pi_cur = pi_cur, pi_next
        tau = n * mu * pi_cur - (n + 1) * pi_prev
        f = (2 * n + 1) / (n * (n + 1))
        S1 += f * (a[n - 1] * pi_cur + b[n - 1] * tau)
        S2 += f * (a[n - 1] * tau + b[n - 1] * pi_cur)
    return S1, S2


def test_single_sphere_s11_matches_mie_phase_function():
    L, k, R, m = 6, 2 * np.pi / 550.0, 240.0, 1.5 + 0.02j
    pos = np.zeros((1, 3))
    t = mie.t_diagonal(L, k, np.array([R]), np.array([m]))
    b_te = t * incident.plane_wave_coeffs(L, k, pos, 0.0, 0.0, 1)
    b_tm = t * incident.plane_wave_coeffs(L, k, pos, 0.0, 0.0, 2)
    betas = np.linspace(0.05, np.pi - 0.05, 23)
    s11 = farfield.s11_azimuthal(L, k, pos, b_te, b_tm, betas, n_alpha=16)
    a, b = mie.bohren_huffman_ab(L, k * R, m)
    S1, S2 = _bh_s1_s2(a, b, betas)
    ref = 0.5 * (np.abs(S1) ** 2 + np.abs(S2) ** 2)
    ratio = s11 / ref
    assert np.max(np.abs(ratio / ratio[0] - 1.0)) < 1e-10
