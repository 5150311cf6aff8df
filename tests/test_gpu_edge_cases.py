"""Edge cases of the batched, BiCGSTAB, near-field, power and S11 entry
points: single spheres (no coupling: b = T a), a batch mixing a one-sphere
ensemble with larger ones, empty point lists, out-of-range RHS indices."""

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


def _ctx(seed, N, L, planes=((0.0, 0.0, 2),)):
    sc = synth.random_cluster(79, seed, N, L, radius=100.0, fill=0.15, n=1.5 + 0.01j)
    c = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, L)
    B.celes_set_incident(c, [B.make_incident("plane", beta=b, alpha=a, pol=p) for (b, a, p) in planes])
    return sc, c


def test_batch_with_a_single_sphere_ensemble():
    ens = [_ctx(0, 1, 3), _ctx(1, 2, 2), _ctx(2, 30, 3, ((0.0, 0.0, 2), (0.5, 1.0, 1)))]
    try:
        bt = B.celes_batch_create([c for _, c in ens])
        try:
            code, infos = B.celes_batch_solve(bt, len(ens), 1e-10, mode=B.CELES_SOLVE_FP64)
            assert code == B.CELES_OK and all(i["residual"] <= 1e-10 for i in infos)
        finally:
            B.celes_batch_destroy(bt)
        for sc, c in ens:
            t = mie.t_diagonal(sc.lmax, sc.k, sc.radii, sc.n_rel)
            got = B.celes_get_coefficients(c)
            planes = ((0.0, 0.0, 2), (0.5, 1.0, 1))
            for r in range(B.celes_num_rhs(c)):
                b, a, p = planes[r]
                ain = incident.plane_wave_coeffs(sc.lmax, sc.k, sc.positions, b, a, p)
                ref = solve.solve_dense(sc.positions, sc.k, sc.lmax, t, ain)
                assert rel(got[r], ref) <= 1e-8
        # one sphere: no coupling at all, b = T a exactly
        sc0, c0 = ens[0]
        t0 = mie.t_diagonal(3, sc0.k, sc0.radii, sc0.n_rel)
        a0 = incident.plane_wave_coeffs(3, sc0.k, sc0.positions, 0.0, 0.0, 2)
        assert rel(B.celes_get_coefficients(c0)[0], t0 * a0) <= 1e-12
    finally:
        for _, c in ens:
            B.celes_destroy(c)


def test_bicgstab_single_sphere_and_tiny_cluster():
    for N in (1, 3):
        sc, c = _ctx(10 + N, N, 2)
        try:
            info = B.celes_solve(c, 1e-12, mode=B.CELES_SOLVE_FP64, solver=B.CELES_SOLVER_BICGSTAB)
            assert info["residual"] <= 1e-12
            t = mie.t_diagonal(2, sc.k, sc.radii, sc.n_rel)
            ain = incident.plane_wave_coeffs(2, sc.k, sc.positions, 0.0, 0.0, 2)
            assert rel(B.celes_get_coefficients(c)[0], solve.solve_dense(sc.positions, sc.k, 2, t, ain)) <= 1e-10
        finally:
            B.celes_destroy(c)


def test_empty_point_list_and_bad_indices():
    sc, c = _ctx(20, 5, 2)
    try:
        B.celes_solve(c, 1e-10, mode=B.CELES_SOLVE_FP64)
        assert B.celes_nearfield(c, np.zeros((0, 3))).shape == (0, 3)
        with pytest.raises(B.CelesError):
            B.celes_nearfield(c, np.ones((2, 3)), rhs=3)
        with pytest.raises(B.CelesError):
            B.celes_s11(c, [0.1, 0.2], rhs_a=0, rhs_b=5)
        with pytest.raises(B.CelesError):
            B.celes_power(c, n_beta=1)
    finally:
        B.celes_destroy(c)


@pytest.mark.parametrize("mode", [B.CELES_SOLVE_FP64, B.CELES_SOLVE_MIXED])
@pytest.mark.parametrize("solver", [B.CELES_SOLVER_GMRES, B.CELES_SOLVER_BICGSTAB])
def test_non_finite_first_iterate_is_a_numeric_error(mode, solver):
    """A NaN user guess makes every residual NaN; the solve must report
    CELES_ENUMERIC instead of reading NaN as converged (a clamp such as
    max(0, NaN) returns 0)."""
    sc, ctx = _ctx(11, 20, 2)
    try:
        B.celes_set_initial_guess(ctx, np.full((1, sc.N, sc.nmax), np.nan + 0j))
        with pytest.raises(B.CelesError) as err:
            B.celes_solve(ctx, 1e-8, mode=mode, x0=B.CELES_X0_USER, use_precond=False, solver=solver)
        assert err.value.code == B.CELES_ENUMERIC
    finally:
        B.celes_destroy(ctx)


def test_resume_from_a_saved_solution():
    """Checkpoint and resume through the custom initial condition: a solve
    stopped at 1e-4 and restarted in a new context from its saved b reaches
    the same answer as a solve from T a, in fewer iterations."""
    sc, ctx = _ctx(12, 40, 3)
    sc2, ctx2 = _ctx(12, 40, 3)
    try:
        B.celes_solve(ctx, 1e-4, mode=B.CELES_SOLVE_FP64, use_precond=False)
        saved = B.celes_get_coefficients(ctx)
        scratch = B.celes_solve(ctx, 1e-10, mode=B.CELES_SOLVE_FP64, use_precond=False, x0=B.CELES_X0_TA)
        b_ref = B.celes_get_coefficients(ctx)
        B.celes_set_initial_guess(ctx2, saved)
        resumed = B.celes_solve(ctx2, 1e-10, mode=B.CELES_SOLVE_FP64, use_precond=False, x0=B.CELES_X0_USER)
        assert resumed["residual"] <= 1e-10 and resumed["guess_used"] >= 1
        assert resumed["iterations"] < scratch["iterations"]
        assert rel(B.celes_get_coefficients(ctx2), b_ref) < 1e-8
    finally:
        B.celes_destroy(ctx)
        B.celes_destroy(ctx2)


def test_preconditioner_too_large_for_the_device_is_enomem():
    """One cuboid holding 3000 spheres at lmax 4 needs 332 GB of FP64 LU
    factors, more than the GPU has: the build fails with CELES_ENOMEM before
    any kernel runs, and the context still solves without it."""
    sc = synth.config2(0, N=3000)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax)
    try:
        B.celes_set_incident(ctx, [B.make_incident("plane", beta=0.0, alpha=0.0, pol=2)])
        with pytest.raises(B.CelesError) as err:
            B.celes_precond_build(ctx, 1.0e7)
        assert err.value.code == B.CELES_ENOMEM
        info = B.celes_solve(ctx, 1e-6, mode=B.CELES_SOLVE_MIXED)
        assert info["residual"] <= 1e-6
    finally:
        B.celes_destroy(ctx)


@pytest.mark.parametrize("kernel", [B.CELES_KERNEL_RTR, B.CELES_KERNEL_DIRECT])
def test_aligned_and_nearly_aligned_pairs(kernel):
    """A cubic lattice (pairs exactly along the axes and diagonals: theta = 0
    or pi, where phi is undefined) and a column of spheres 0, 1e-3 and 1e-6 nm
    off the z axis: both precisions against the oracle's dense W."""
    from oracle import translation
    g = np.arange(3) * 250.0
    lattice = np.array([[x, y, z] for x in g for y in g for z in g])
    column = np.array([[800.0 + dx, 0.0, 260.0 * q] for q, dx in enumerate([0.0, 1e-3, 1e-6, 0.0, 2e-3])])
    pos = np.concatenate([lattice, column])
    N, L = len(pos), 4
    radii = np.full(N, 100.0)
    k0 = 2.0 * np.pi / 550.0
    ctx = B.celes_create(pos, radii, np.full(N, 1.5 + 0.01j), 1.0, k0, L, kernel=kernel)
    try:
        nmax = 2 * L * (L + 2)
        x = synth.random_vector(2, 91, (N, nmax))
        ref = (translation.coupling_matrix(pos, k0, L) @ x.reshape(-1)).reshape(N, nmax)
        for precision, dt, tol in [(B.CELES_FP64, torch.complex128, 1e-10), (B.CELES_FP32, torch.complex64, 1e-5)]:
            xd = torch.from_numpy(x).to(dt).cuda()
            yd = torch.zeros_like(xd)
            B.celes_coupling_matvec(ctx, xd, yd, precision=precision)
            torch.cuda.synchronize()
            y = yd.cpu().numpy().astype(np.complex128)
            assert np.all(np.isfinite(y))
            assert rel(y, ref) < tol, (precision, rel(y, ref))
    finally:
        B.celes_destroy(ctx)
