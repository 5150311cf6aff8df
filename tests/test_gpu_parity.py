"""GPU parity: every step of the CUDA path against the FP64 CPU oracle, on the
same seeded inputs, through the C ABI.

Tolerances (relative L2 unless stated):
  * FP64 kernels (T-matrix, incident coefficients, FP64 coupling / master
    matvec, preconditioner apply, far field): 1e-10 (the FP64 requirement);
    the arithmetic itself lands near 1e-14.
  * FP32 coupling / master matvec: 1e-5 (the chosen-form requirement).
  * Solves: FP64 GMRES to 1e-12 -> 1e-10 of the dense LU solution;
    mixed FP32 + FP64 refinement to 1e-6 -> 1e-5.
"""

import numpy as np
import pytest

import synth
from oracle import farfield, incident, mie, precond, solve, translation

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


def make_ctx(sc, **kw):
    return B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax, **kw)


def dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x).astype(dtype)).cuda()


def gpu_matvec(ctx, x, precision, master=False, nrhs=1):
    dt = np.complex128 if precision == B.CELES_FP64 else np.complex64
    xd = dev(x, dt)
    yd = torch.zeros_like(xd)
    fn = B.celes_master_matvec if master else B.celes_coupling_matvec
    fn(ctx, xd, yd, nrhs=nrhs, precision=precision)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128)


CLUSTERS = [
    # (N, L, polydisperse, n)
    (1, 3, False, 1.52 + 0j),
    (2, 2, False, 1.5 + 0.01j),
    (33, 1, False, 1.6 + 0j),
    (50, 3, False, 1.52 + 0j),
    (37, 2, True, 1.45 + 0.02j),
    (29, 4, True, 1.5 + 0.001j),
    (21, 5, False, 1.8 + 0j),
]


@pytest.mark.parametrize("N,L,poly,n", CLUSTERS)
def test_tmatrix_and_plane_wave(N, L, poly, n):
    sc = synth.random_cluster(21, N + L, N, L, radius=110.0, fill=0.2, n=n, polydisperse=poly)
    ctx = make_ctx(sc)
    try:
        t_ref = mie.t_diagonal(L, sc.k, sc.radii, sc.n_rel)
        assert rel(B.celes_get_tmatrix(ctx), t_ref) < 1e-12
        incs = [B.make_incident("plane", beta=0.0, alpha=0.0, pol=2),
                B.make_incident("plane", beta=0.7, alpha=-1.1, pol=1, E0=0.3 - 0.4j)]
        B.celes_set_incident(ctx, incs)
        a = B.celes_get_incident_coefficients(ctx)
        a0 = incident.plane_wave_coeffs(L, sc.k, sc.positions, 0.0, 0.0, 2)
        a1 = (0.3 - 0.4j) * incident.plane_wave_coeffs(L, sc.k, sc.positions, 0.7, -1.1, 1)
        assert rel(a[0], a0) < 1e-12 and rel(a[1], a1) < 1e-12
    finally:
        B.celes_destroy(ctx)


@pytest.mark.parametrize("n", [1.5 + 0.05j, 2.0 + 0.3j, 1.33 + 1e-3j, 1.7 + 0j])
def test_tmatrix_at_large_size_parameters(n):
    # the FP64 Mie kernel (App. B) at size parameters k R = 4 .. 30 with
    # absorbing and lossless spheres, entry by entry against the oracle
    k0 = 2 * np.pi / 550.0
    radii = np.array([4.0, 10.0, 22.0, 30.0]) / k0
    pos = np.zeros((4, 3))
    pos[:, 0] = np.arange(4) * 6000.0
    ctx = B.celes_create(pos, radii, np.full(4, n), 1.0, k0, 5)
    try:
        t = B.celes_get_tmatrix(ctx)
        ref = mie.t_diagonal(5, k0, radii, np.full(4, n))
        assert np.max(np.abs(t - ref) / np.abs(ref)) < 1e-10
    finally:
        B.celes_destroy(ctx)


def test_gaussian_beam_far_from_the_axis_of_the_slab():
    # the 10 000-sphere slab with its 2 um Gaussian beam: the 20 spheres
    # farthest from the beam axis (k rho ~ 100, where the coefficients are
    # ~1e-8 of the peak) and 20 at the median distance, with the bench's
    # 128-node beta rule.  Errors are measured against the beam's peak
    # coefficient (the on-axis sphere), since far out the coefficients are
    # cancellation-limited to ~1e-15 of the peak in any FP64 evaluation.
    sc = synth.config2(0)
    rho = np.hypot(sc.positions[:, 0], sc.positions[:, 1])
    order = np.argsort(-rho)
    sel = np.concatenate([order[:20], order[sc.N // 2:sc.N // 2 + 20], order[-1:]])
    inc = sc.incidents[0]
    ctx = B.celes_create(sc.positions[sel], sc.radii[sel], sc.n_sphere[sel], sc.n0, sc.k0, sc.lmax)
    try:
        B.celes_set_incident(ctx, [B.make_incident("gaussian", waist=inc.waist, focus=inc.focus,
                                                   alpha_G=inc.alpha_G, n_beta=128)])
        a = B.celes_get_incident_coefficients(ctx)[0]
        ref = incident.gaussian_beam_coeffs(sc.lmax, sc.k, sc.positions[sel], inc.waist, inc.focus, inc.alpha_G,
                                            n_beta=128)
        peak = np.max(np.abs(ref[-1]))
        assert np.max(np.abs(a - ref)) < 1e-12 * peak
        assert rel(a[20:40], ref[20:40]) < 1e-8   # ~1e-4 of the peak: cancellation-limited near 1e-11
        assert rel(a[:20], ref[:20]) < 1e-5       # ~1e-8 of the peak: 128 vs 256 nodes differ by 3e-8
    finally:
        B.celes_destroy(ctx)


def test_gaussian_beam_coefficients():
    sc = synth.random_cluster(22, 0, 24, 3, radius=120.0, fill=0.15, n=1.5 + 0.001j)
    ctx = make_ctx(sc)
    try:
        focus = (float(sc.positions[:, 0].mean()) + 50.0, float(sc.positions[:, 1].mean()) - 30.0,
                 float(sc.positions[:, 2].min()))
        B.celes_set_incident(ctx, [B.make_incident("gaussian", waist=1000.0, focus=focus, alpha_G=-np.pi / 2,
                                                   n_beta=96)])
        a = B.celes_get_incident_coefficients(ctx)[0]
        ref = incident.gaussian_beam_coeffs(3, sc.k, sc.positions, 1000.0, focus, -np.pi / 2, n_beta=96)
        assert rel(a, ref) < 1e-10
    finally:
        B.celes_destroy(ctx)


@pytest.mark.parametrize("kernel", [B.CELES_KERNEL_RTR, B.CELES_KERNEL_DIRECT])
@pytest.mark.parametrize("N,L,poly,n", CLUSTERS)
def test_coupling_and_master_matvec(N, L, poly, n, kernel):
    sc = synth.random_cluster(23, N + L, N, L, radius=100.0, fill=0.25, n=n, polydisperse=poly)
    ctx = make_ctx(sc, kernel=kernel)
    try:
        W = translation.coupling_matrix(sc.positions, sc.k, L)
        t = mie.t_diagonal(L, sc.k, sc.radii, sc.n_rel)
        x = synth.random_vector(23, 100 + N, (sc.N, sc.nmax))
        y_ref = (W @ x.reshape(-1)).reshape(x.shape)
        m_ref = solve.apply_M(W, t, x)
        y64 = gpu_matvec(ctx, x, B.CELES_FP64)
        m64 = gpu_matvec(ctx, x, B.CELES_FP64, master=True)
        y32 = gpu_matvec(ctx, x, B.CELES_FP32)
        m32 = gpu_matvec(ctx, x, B.CELES_FP32, master=True)
        if N == 1:
            assert np.all(y64 == 0) and np.all(y32 == 0)
            assert rel(m64, x) == 0.0
            return
        assert rel(y64, y_ref) < 1e-10
        assert rel(m64, m_ref) < 1e-10
        assert rel(y32, y_ref) < 1e-5
        assert rel(m32, m_ref) < 1e-5
    finally:
        B.celes_destroy(ctx)


def test_multi_rhs_matvec_and_chunking():
    sc = synth.random_cluster(24, 0, 70, 3, radius=90.0, fill=0.2)
    W = translation.coupling_matrix(sc.positions, sc.k, 3)
    x = synth.random_vector(24, 1, (3, sc.N, sc.nmax))
    ref = np.stack([(W @ x[r].reshape(-1)).reshape(sc.N, sc.nmax) for r in range(3)])
    for chunks, kernel in ((0, B.CELES_KERNEL_AUTO), (1, B.CELES_KERNEL_RTR), (3, B.CELES_KERNEL_DIRECT),
                           (7, B.CELES_KERNEL_RTR)):
        ctx = make_ctx(sc, chunks=chunks, kernel=kernel)
        try:
            assert rel(gpu_matvec(ctx, x, B.CELES_FP64, nrhs=3), ref) < 1e-10
            assert rel(gpu_matvec(ctx, x, B.CELES_FP32, nrhs=3), ref) < 1e-5
        finally:
            B.celes_destroy(ctx)


def _dense_reference(sc, a):
    t = mie.t_diagonal(sc.lmax, sc.k, sc.radii, sc.n_rel)
    return solve.solve_dense(sc.positions, sc.k, sc.lmax, t, a), t


def test_config1_fp64_solve_matches_dense_lu():
    sc = synth.config1(0)
    ctx = make_ctx(sc)
    try:
        B.celes_set_incident(ctx, [B.make_incident("plane", beta=0.0, alpha=0.0, pol=2)])
        info = B.celes_solve(ctx, 1e-12, mode=B.CELES_SOLVE_FP64)
        b = B.celes_get_coefficients(ctx)[0]
        a = incident.plane_wave_coeffs(3, sc.k, sc.positions, 0.0, 0.0, 2)
        ref, _ = _dense_reference(sc, a)
        assert info["residual"] <= 1e-12
        assert rel(b, ref) < 1e-10
        # the tolerance the workload names (1e-10) also gives 1e-9 coefficients
        B.celes_solve(ctx, 1e-10, mode=B.CELES_SOLVE_FP64)
        assert rel(B.celes_get_coefficients(ctx)[0], ref) < 1e-8
    finally:
        B.celes_destroy(ctx)


def test_config1_mixed_solve_reaches_chosen_form_accuracy():
    sc = synth.config1(0)
    ctx = make_ctx(sc)
    try:
        B.celes_set_incident(ctx, [B.make_incident("plane", beta=0.0, alpha=0.0, pol=2)])
        info = B.celes_solve(ctx, 1e-6, mode=B.CELES_SOLVE_MIXED)
        b = B.celes_get_coefficients(ctx)[0]
        a = incident.plane_wave_coeffs(3, sc.k, sc.positions, 0.0, 0.0, 2)
        ref, t = _dense_reference(sc, a)
        assert info["residual"] <= 1e-6
        assert info["matvecs_fp32"] > info["matvecs_fp64"] >= 1
        assert rel(b, ref) < 1e-5
        # the reported residual is the FP64 one
        W = translation.coupling_matrix(sc.positions, sc.k, 3)
        r = (t * a).reshape(-1) - solve.apply_M(W, t, b).reshape(-1)
        assert np.linalg.norm(r) / np.linalg.norm((t * a).reshape(-1)) <= 1.01e-6
    finally:
        B.celes_destroy(ctx)


@pytest.mark.parametrize("N,L,edge", [(120, 3, 700.0), (90, 3, 450.0), (60, 4, 1e5), (33, 5, 380.0)])
def test_preconditioner_apply_large_blocks(N, L, edge):
    # blocks of several 32-row tiles with a ragged last tile: the cluster form
    # of the apply (2 or 4 CTAs per block), two right-hand sides, in place and
    # out of place, against the oracle's block solves
    sc = synth.random_cluster(26, N + L, N, L, radius=100.0, fill=0.3, n=1.55 + 0.01j)
    ctx = make_ctx(sc)
    try:
        t = mie.t_diagonal(L, sc.k, sc.radii, sc.n_rel)
        B.celes_precond_build(ctx, edge)
        nb, maxd, ent = B.celes_precond_stats(ctx)
        assert maxd >= 96
        P = precond.BlockPreconditioner(sc.positions, sc.k, L, t, edge)
        y = synth.random_vector(26, N, (2, sc.N, sc.nmax))
        ref = np.stack([P.apply(y[0]), P.apply(y[1])])
        for prec, dt, tol in ((B.CELES_FP64, np.complex128, 1e-10), (B.CELES_FP32, np.complex64, 1e-5)):
            yd = dev(y, dt)
            xd = torch.full_like(yd, float("nan"))
            B.celes_precond_apply(ctx, yd, xd, nrhs=2, precision=prec)
            torch.cuda.synchronize()
            assert rel(xd.cpu().numpy(), ref) < tol
            B.celes_precond_apply(ctx, yd, yd, nrhs=2, precision=prec)
            torch.cuda.synchronize()
            assert rel(yd.cpu().numpy(), ref) < tol
    finally:
        B.celes_destroy(ctx)


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("N,L,poly,n", CLUSTERS)
def test_coupling_alternative_fp32_shape(N, L, poly, n, variant):
    # the autotuner's other FP32 launch shapes, forced, against the dense W:
    # the alternative compile-time shape (bit 0), the cluster reduction of the
    # partial sums (bit 1), their reduction in L2 (bit 2), and combinations
    sc = synth.random_cluster(23, N + L, N, L, radius=100.0, fill=0.25, n=n, polydisperse=poly)
    ctx = make_ctx(sc, variant=variant)
    try:
        W = translation.coupling_matrix(sc.positions, sc.k, L)
        x = synth.random_vector(23, 200 + N, (sc.N, sc.nmax))
        y_ref = (W @ x.reshape(-1)).reshape(x.shape)
        y = gpu_matvec(ctx, x, B.CELES_FP32)
        if N == 1:
            assert np.all(y == 0)
        else:
            assert rel(y, y_ref) < 1e-5
        v, ch, _ = B.celes_coupling_shape(ctx, B.CELES_FP32)
        assert v == variant and ch >= 1
        if variant & 2:  # the FP64 kernel takes the cluster reduction too
            y64 = gpu_matvec(ctx, x, B.CELES_FP64)
            if N == 1:
                assert np.all(y64 == 0)
            else:
                assert rel(y64, y_ref) < 1e-10
    finally:
        B.celes_destroy(ctx)


@pytest.mark.parametrize("N,L,variant", [(333, 3, 2), (700, 4, 2), (700, 4, 3), (517, 5, 3), (450, 2, 2),
                                         (333, 3, 4), (700, 4, 4), (700, 4, 6), (517, 5, 5), (517, 5, 7),
                                         (450, 2, 4), (450, 1, 6)])
def test_coupling_cluster_reduction_on_sampled_rows(N, L, variant):
    # enough spheres for several source chunks per receiver block, so that the
    # partial sums really are added in clusters of CTAs or in L2; ragged block
    # counts
    sc = synth.config2(0, N=N, lmax=L)
    ctx = make_ctx(sc, variant=variant)
    try:
        x = synth.random_vector(27, N + L, (sc.N, sc.nmax))
        rows = [0, 1, N // 3, N // 2 + 1, N - 2, N - 1]
        ref = translation.coupling_matvec_rows(sc.positions, sc.k, L, x, rows)
        y32 = gpu_matvec(ctx, x, B.CELES_FP32)
        _, ch, _ = B.celes_coupling_shape(ctx, B.CELES_FP32)
        assert ch >= 4 and ch % 4 == 0
        assert rel(y32[rows], ref) < 1e-5
        y64 = gpu_matvec(ctx, x, B.CELES_FP64)
        assert rel(y64[rows], ref) < 1e-10
    finally:
        B.celes_destroy(ctx)


@pytest.mark.parametrize("L", [3, 4])
def test_autotuner_picks_a_shape_and_keeps_the_result(L):
    # the tuned context and an untuned one give the same product (to FP32
    # rounding), and the tuned shape is reported
    sc = synth.config2(0, N=1500, lmax=L)
    x = synth.random_vector(24, L, (sc.N, sc.nmax))
    c1 = make_ctx(sc)
    c0 = make_ctx(sc, autotune=False)
    try:
        y1 = gpu_matvec(c1, x, B.CELES_FP32)
        y0 = gpu_matvec(c0, x, B.CELES_FP32)
        assert rel(y1, y0) < 1e-5
        v, ch, ms = B.celes_coupling_shape(c1, B.CELES_FP32)
        assert v in range(8) and ch >= 1 and ms > 0
        v0, ch0, ms0 = B.celes_coupling_shape(c0, B.CELES_FP32)
        assert v0 == 0 and ms0 == 0
        rows = [0, 700, sc.N - 1]
        ref = translation.coupling_matvec_rows(sc.positions, sc.k, L, x, rows)
        assert rel(y1[rows], ref) < 1e-5
    finally:
        B.celes_destroy(c1)
        B.celes_destroy(c0)


def test_preconditioner_apply_and_preconditioned_solve():
    sc = synth.random_cluster(25, 0, 40, 2, radius=100.0, fill=0.3, n=1.6 + 0.01j)
    ctx = make_ctx(sc)
    try:
        t = mie.t_diagonal(2, sc.k, sc.radii, sc.n_rel)
        edge = 300.0
        B.celes_precond_build(ctx, edge)
        P = precond.BlockPreconditioner(sc.positions, sc.k, 2, t, edge)
        y = synth.random_vector(25, 2, (sc.N, sc.nmax))
        ref = P.apply(y)
        for prec, dt, tol in ((B.CELES_FP64, np.complex128, 1e-10), (B.CELES_FP32, np.complex64, 1e-5)):
            yd = dev(y, dt)
            xd = torch.zeros_like(yd)
            B.celes_precond_apply(ctx, yd, xd, precision=prec)
            torch.cuda.synchronize()
            assert rel(xd.cpu().numpy(), ref) < tol
        # in place
        yd = dev(y, np.complex128)
        B.celes_precond_apply(ctx, yd, yd, precision=B.CELES_FP64)
        torch.cuda.synchronize()
        assert rel(yd.cpu().numpy(), ref) < 1e-10
        B.celes_set_incident(ctx, [B.make_incident("plane", beta=0.2, alpha=0.4, pol=1)])
        a = incident.plane_wave_coeffs(2, sc.k, sc.positions, 0.2, 0.4, 1)
        ref_b, _ = _dense_reference(sc, a)
        info_p = B.celes_solve(ctx, 1e-11, mode=B.CELES_SOLVE_FP64, use_precond=True)
        assert rel(B.celes_get_coefficients(ctx)[0], ref_b) < 1e-9
        info_n = B.celes_solve(ctx, 1e-11, mode=B.CELES_SOLVE_FP64, use_precond=False)
        assert info_p["iterations"] < info_n["iterations"]
        info_m = B.celes_solve(ctx, 1e-6, mode=B.CELES_SOLVE_MIXED, use_precond=True)
        assert info_m["residual"] <= 1e-6 and rel(B.celes_get_coefficients(ctx)[0], ref_b) < 1e-5
    finally:
        B.celes_destroy(ctx)


def test_farfield_matches_oracle_and_optical_theorem():
    sc = synth.random_cluster(26, 0, 20, 3, radius=100.0, fill=0.2, n=1.5 + 0.05j)
    ctx = make_ctx(sc)
    try:
        B.celes_set_incident(ctx, [B.make_incident("plane", beta=0.3, alpha=0.8, pol=2)])
        B.celes_solve(ctx, 1e-12, mode=B.CELES_SOLVE_FP64)
        b = B.celes_get_coefficients(ctx)[0]
        rng = np.random.default_rng(3)
        dirs = np.stack([np.arccos(rng.uniform(-1, 1, 40)), rng.uniform(0, 2 * np.pi, 40)], axis=1)
        g = B.celes_farfield(ctx, dirs)
        assert rel(g, farfield.farfield_amplitude(3, sc.k, sc.positions, b, dirs)) < 1e-10
        # optical theorem on GPU results: C_ext from the forward amplitude of
        # the GPU far field = C_sca (quadrature of |g|^2) + C_abs
        a = B.celes_get_incident_coefficients(ctx)[0]
        t = B.celes_get_tmatrix(ctx)
        gf = B.celes_farfield(ctx, [[0.3, 0.8]])[0]
        ce = -8 * np.pi ** 2 / sc.k ** 2 * np.real(gf[1])
        assert abs(ce - solve.c_ext(sc.k, a, b)) < 1e-9 * ce
        xg, wg = np.polynomial.legendre.leggauss(40)
        al = 2 * np.pi * np.arange(80) / 80
        Bt, At = np.meshgrid(np.arccos(-xg), al, indexing="ij")
        gg = B.celes_farfield(ctx, np.stack([Bt.ravel(), At.ravel()], axis=1))
        I = np.sum(np.abs(gg) ** 2, axis=1).reshape(40, 80)
        cs = 4 * np.pi ** 2 / sc.k ** 2 * np.sum(wg[:, None] * I) * (2 * np.pi / 80)
        assert abs(ce - (cs + solve.c_abs(sc.k, t, b))) < 1e-8 * ce
    finally:
        B.celes_destroy(ctx)


def test_full_size_config2_sampled_rows():
    """The bench workload (10 000 polydisperse spheres, lmax 4) in the launch
    configuration the bench times: sampled receivers against the oracle's
    on-the-fly rows."""
    sc = synth.config2(0)
    ctx = make_ctx(sc)
    ctx_d = make_ctx(sc, kernel=B.CELES_KERNEL_DIRECT)
    try:
        x = synth.random_vector(2, 77, (sc.N, sc.nmax))
        y64 = gpu_matvec(ctx, x, B.CELES_FP64)
        y32 = gpu_matvec(ctx, x, B.CELES_FP32)
        y32d = gpu_matvec(ctx_d, x, B.CELES_FP32)
        rows = list(np.random.default_rng(5).choice(sc.N, 8, replace=False))
        ref = translation.coupling_matvec_rows(sc.positions, sc.k, sc.lmax, x, rows)
        assert rel(y64[rows], ref) < 1e-10
        assert rel(y32[rows], ref) < 1e-5
        assert rel(y32d[rows], ref) < 1e-5
        # the two FP32 kernels agree on every receiver
        assert rel(y32, y64) < 1e-5 and rel(y32d, y64) < 1e-5
    finally:
        B.celes_destroy(ctx)
        B.celes_destroy(ctx_d)


def test_maximum_size_config5_sampled_rows():
    """The largest workload (100 000 monodisperse spheres in a 4 um slab,
    lmax 3, 1e10 ordered pairs) through the FP32 kernel in its default launch
    shape: sampled receivers against the oracle's on-the-fly FP64 rows."""
    sc = synth.config5(0)
    ctx = make_ctx(sc)
    try:
        x = synth.random_vector(2, 78, (sc.N, sc.nmax))
        y32 = gpu_matvec(ctx, x, B.CELES_FP32)
        assert np.all(np.isfinite(y32))
        rows = [0, sc.N - 1] + [int(r) for r in np.random.default_rng(6).choice(sc.N, 2, replace=False)]
        ref = translation.coupling_matvec_rows(sc.positions, sc.k, sc.lmax, x, rows)
        assert rel(y32[rows], ref) < 1e-5
    finally:
        B.celes_destroy(ctx)


def test_overlap_and_argument_errors():
    pos = np.array([[0.0, 0.0, 0.0], [150.0, 0.0, 0.0]])
    with pytest.raises(B.CelesError) as e:
        B.celes_create(pos, [100.0, 100.0], [1.5, 1.5], 1.0, 2 * np.pi / 550, 3)
    assert e.value.code == B.CELES_EOVERLAP
    sc = synth.random_cluster(27, 0, 5, 2)
    ctx = make_ctx(sc)
    try:
        with pytest.raises(B.CelesError) as e:
            B.celes_solve(ctx, 1e-6)
        assert e.value.code == B.CELES_ESTATE
        B.celes_set_incident(ctx, [B.make_incident("plane")])
        x = dev(np.zeros((sc.N, sc.nmax)), np.complex128)
        with pytest.raises(B.CelesError) as e:
            B.celes_coupling_matvec(ctx, x, x)
        assert e.value.code == B.CELES_EINVAL
        # iteration budget exhausted: ENOCONV with the best iterate kept
        info = B.celes_solve(ctx, 1e-14, mode=B.CELES_SOLVE_FP64, max_iter=1, raise_on_noconv=False)
        assert info["status"] == B.CELES_ENOCONV
        assert np.all(np.isfinite(B.celes_get_coefficients(ctx)))
    finally:
        B.celes_destroy(ctx)
