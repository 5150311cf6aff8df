"""The oracle reproduces its stored values (tests/golden/oracle_regression.json)
to 1e-12 relative: a guard against unintended changes of the oracle."""

import json
import os

import numpy as np

import synth
from oracle import incident, mie, solve, translation

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_regression.json")


def _c(v):
    a = np.asarray(v, dtype=float)
    return a[:, 0] + 1j * a[:, 1]


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def test_oracle_matches_stored_values():
    with open(GOLDEN) as fh:
        g = json.load(fh)
    k = 2 * np.pi / 550.0
    radii = np.array([100.0, 150.0, 60.0])
    n_rel = np.array([1.52 + 0j, 1.5 + 0.01j, 2.0 + 0.5j])
    assert _rel(mie.t_diagonal(3, k, radii, n_rel), _c(g["mie_t_diagonal_L3"])) < 1e-12
    pos = np.array([[0.0, 0.0, 0.0], [180.0, -90.0, 240.0]])
    assert _rel(translation.coupling_matrix(pos, k, 2)[:16, 16:], _c(g["coupling_block_L2"])) < 1e-12
    sc = synth.random_cluster(61, 0, 4, 2, radius=100.0, fill=0.2, n=1.5 + 0.02j)
    assert np.allclose(sc.positions, np.array(g["cluster4_positions"]), rtol=0, atol=1e-9)
    t = mie.t_diagonal(2, sc.k, sc.radii, sc.n_rel)
    a = incident.plane_wave_coeffs(2, sc.k, sc.positions, 0.4, 0.7, 1)
    assert _rel(solve.solve_dense(sc.positions, sc.k, 2, t, a), _c(g["cluster4_solution_L2"])) < 1e-12
