"""The package-level Python API (Simulation, BatchSolver, LearnedGuess) on a
small Gaussian-beam cluster: the user-facing flow gives the same numbers as
the oracle (solves vs dense LU, energy balance R + T = 1 for lossless
spheres, near field vs the oracle's SVWF sum)."""

import numpy as np
import pytest

import synth
from oracle import incident, mie, solve, svwf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_02145_gb300 as P  # noqa: E402
from paper_1706_02145_gb300 import binding as B  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    B.load()


def test_simulation_flow():
    sc = synth.random_cluster(89, 0, 14, 3, radius=110.0, fill=0.15, n=1.6 + 0j)
    sim = P.Simulation.from_scene(sc)
    try:
        w, focus, aG = 1400.0, (0.0, 0.0, 0.0), -np.pi / 2
        sim.set_incident([synth.Incident("gaussian", waist=w, focus=focus, alpha_G=aG),
                          synth.Incident("plane", beta=0.0, alpha=0.0, pol=1),
                          synth.Incident("plane", beta=0.0, alpha=0.0, pol=2)], n_beta=256)
        sim.precond_build(500.0)
        info = sim.solve(1e-11, mode=P.CELES_SOLVE_FP64, solver=P.CELES_SOLVER_BICGSTAB)
        assert info["residual"] <= 1e-11
        b = sim.coefficients()
        t = mie.t_diagonal(3, sc.k, sc.radii, sc.n_rel)
        a = incident.plane_wave_coeffs(3, sc.k, sc.positions, 0.0, 0.0, 1)
        assert rel(b[1], solve.solve_dense(sc.positions, sc.k, 3, t, a)) <= 1e-9
        R, T = sim.power(0, n_beta=96, n_alpha=96)
        assert abs(R + T - 1.0) < 1e-7
        s = sim.s11(np.linspace(0.0, np.pi, 7), 1, 2)
        assert np.all(s > 0)
        pts = np.array([[3000.0, -2000.0, 500.0], [-2500.0, 1000.0, -800.0]])
        E = sim.nearfield(pts, rhs=1, what=0)
        ref = sum(svwf.field_expansion(3, b[1][i], 3, sc.k, pts, origin=sc.positions[i]) for i in range(sc.N))
        assert rel(E, ref) <= 1e-10
    finally:
        sim.close()


def test_batch_solver_and_learned_guess_wrappers():
    sims = []
    try:
        for q, (N, L) in enumerate([(20, 2), (35, 3)]):
            sc = synth.random_cluster(89, 10 + q, N, L, radius=100.0, fill=0.15, n=1.5 + 0.01j)
            s = P.Simulation.from_scene(sc)
            s.set_incident([synth.Incident("plane", beta=0.2, alpha=0.1, pol=2)])
            sims.append((sc, s))
        bs = P.BatchSolver([s for _, s in sims])
        try:
            code, infos = bs.solve(1e-8, mode=P.CELES_SOLVE_MIXED)
            assert code == B.CELES_OK and all(i["residual"] <= 1e-8 for i in infos)
        finally:
            bs.close()
        sc, s = sims[1]
        g = P.LearnedGuess(3, width=32, layers=2, seed=1)
        try:
            l0 = g.train(s, steps=0)
            for _ in range(20):
                g.train(s, steps=1, lr=3e-3)
            assert g.train(s, steps=0) < l0
            s.predict_guess(g)
            info = s.solve(1e-8, mode=P.CELES_SOLVE_MIXED, x0=P.CELES_X0_LEARNED)
            assert info["residual"] <= 1e-8
        finally:
            g.close()
    finally:
        for _, s in sims:
            s.close()
