"""Write oracle_regression.json: values of the FP64 oracle on small fixed
inputs, so that any later change to the oracle's arithmetic shows up as a
failing test (tests/test_oracle_regression.py) and has to be justified.

The paper prints no worked numerical example that this build can reproduce
(its validation cases use packings that are not published), so these values
are the oracle's own; the oracle itself is pinned by closed forms,
identities and brute force in the other oracle tests.

Calls only oracle/ and synth/:  python tests/golden/make_oracle_regression.py
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import incident, mie, solve, translation  # noqa: E402


def cplx(a):
    a = np.asarray(a, dtype=complex).ravel()
    return [[float(v.real), float(v.imag)] for v in a]


def main():
    out = {}
    # Mie T-matrix diagonal (App. B) for three spheres
    k = 2 * np.pi / 550.0
    radii = np.array([100.0, 150.0, 60.0])
    n_rel = np.array([1.52 + 0j, 1.5 + 0.01j, 2.0 + 0.5j])
    out["mie_t_diagonal_L3"] = cplx(mie.t_diagonal(3, k, radii, n_rel))
    # one coupling block (Sec. 3.2.2, a5/b5 form) at a fixed separation
    d = np.array([180.0, -90.0, 240.0])
    pos = np.array([[0.0, 0.0, 0.0], d])
    out["coupling_block_L2"] = cplx(translation.coupling_matrix(pos, k, 2)[:16, 16:])
    # dense solution of a 4-sphere cluster under an oblique plane wave
    sc = synth.random_cluster(61, 0, 4, 2, radius=100.0, fill=0.2, n=1.5 + 0.02j)
    t = mie.t_diagonal(2, sc.k, sc.radii, sc.n_rel)
    a = incident.plane_wave_coeffs(2, sc.k, sc.positions, 0.4, 0.7, 1)
    out["cluster4_positions"] = sc.positions.tolist()
    out["cluster4_solution_L2"] = cplx(solve.solve_dense(sc.positions, sc.k, 2, t, a))
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as fh:
        json.dump(out, fh, indent=0)


if __name__ == "__main__":
    main()
