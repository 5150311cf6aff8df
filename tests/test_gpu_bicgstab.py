"""BiCGSTAB (the second Krylov solver the paper names, Sec. 3.2) through the
same solve entry point: FP64 to 1e-12 reaches the oracle's dense-LU solution
to 1e-10; FP32 inner + FP64 refinement to 1e-6 reaches it to 1e-5; with and
without the block preconditioner; several RHS."""

import numpy as np
import pytest

import synth
from oracle import incident, mie, solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


PLANES = [(0.0, 0.0, 2), (0.7, 1.3, 1)]


@pytest.mark.parametrize("seed,N,L,precond", [(0, 40, 3, False), (1, 120, 2, True), (2, 25, 4, False)])
@pytest.mark.parametrize("mode,tol,bound", [(B.CELES_SOLVE_FP64, 1e-12, 1e-10), (B.CELES_SOLVE_MIXED, 1e-6, 1e-5)])
def test_bicgstab_matches_dense_lu(seed, N, L, precond, mode, tol, bound):
    sc = synth.random_cluster(47, seed, N, L, radius=100.0, fill=0.2, n=1.55 + 0.01j, polydisperse=True)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, L)
    try:
        B.celes_set_incident(ctx, [B.make_incident("plane", beta=b, alpha=a, pol=p) for (b, a, p) in PLANES])
        if precond:
            B.celes_precond_build(ctx, 400.0)
        info = B.celes_solve(ctx, tol, mode=mode, solver=B.CELES_SOLVER_BICGSTAB, use_precond=precond)
        assert info["residual"] <= tol
        assert info["iterations"] > 0
        got = B.celes_get_coefficients(ctx)
        t = mie.t_diagonal(L, sc.k, sc.radii, sc.n_rel)
        for r, (b, a, p) in enumerate(PLANES):
            ain = incident.plane_wave_coeffs(L, sc.k, sc.positions, b, a, p)
            ref = solve.solve_dense(sc.positions, sc.k, L, t, ain)
            assert rel(got[r], ref) <= bound
    finally:
        B.celes_destroy(ctx)


def test_unknown_solver_rejected():
    sc = synth.random_cluster(47, 9, 10, 2, radius=100.0, fill=0.2)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, 2)
    try:
        B.celes_set_incident(ctx, [B.make_incident("plane")])
        with pytest.raises(B.CelesError):
            B.celes_solve(ctx, 1e-6, solver=7)
    finally:
        B.celes_destroy(ctx)
