"""Batched lockstep solves over uneven ensembles (several lmax, sizes and RHS).

1. The batched operator (one persistent coupling launch per lmax, graph
   replay, batched epilogue) against the oracle's master operator
   x - T (W x) per system: FP64 1e-10, FP32 1e-5 relative L2.
2. The batched mixed-precision solve reaches tol = 1e-6 on every system and
   the dense LU solution of the oracle to 1e-5; the FP64 batched solve to
   1e-11 reaches it to 1e-9.
3. A batch that lets systems converge at different iterations (masking) gives
   the same answers as solving them one by one.
"""

import numpy as np
import pytest

import synth
from oracle import incident, mie, solve, translation

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


# (seed, N, lmax, number of plane waves): uneven sizes, every lmax of the batch kernels
ENSEMBLES = [(0, 37, 2, 2), (1, 90, 3, 1), (2, 21, 5, 1), (3, 64, 1, 3), (4, 50, 4, 2)]
PLANES = [(0.0, 0.0, 2), (0.4, 0.3, 1), (1.1, 2.0, 2)]


def _ensemble(seed, N, L, nrhs):
    sc = synth.random_cluster(43, seed, N, L, radius=90.0, fill=0.15, n=1.5 + 0.02j, polydisperse=True)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, L)
    B.celes_set_incident(ctx, [B.make_incident("plane", beta=b, alpha=a, pol=p) for (b, a, p) in PLANES[:nrhs]])
    return sc, ctx


@pytest.fixture(scope="module")
def batch_setup():
    ens = [_ensemble(*e) for e in ENSEMBLES]
    yield ens
    for _, ctx in ens:
        B.celes_destroy(ctx)


def _references(ens):
    out = []
    for (sc, ctx), (_, N, L, nrhs) in zip(ens, ENSEMBLES):
        t = mie.t_diagonal(L, sc.k, sc.radii, sc.n_rel)
        for (b, a, p) in PLANES[:nrhs]:
            ain = incident.plane_wave_coeffs(L, sc.k, sc.positions, b, a, p)
            out.append(solve.solve_dense(sc.positions, sc.k, L, t, ain))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_operator_matches_oracle(batch_setup, precision):
    ens = batch_setup
    b = B.celes_batch_create([c for _, c in ens])
    try:
        n = B.celes_batch_num_unknowns(b)
        assert B.celes_batch_num_systems(b) == sum(e[3] for e in ENSEMBLES)
        rng = np.random.default_rng(5)
        x = rng.normal(size=n) + 1j * rng.normal(size=n)
        dt = torch.complex128 if precision == "fp64" else torch.complex64
        prec = B.CELES_FP64 if precision == "fp64" else B.CELES_FP32
        xd = torch.from_numpy(x).to(dt).cuda()
        yd = torch.zeros_like(xd)
        B.celes_batch_master_matvec(b, xd, yd, precision=prec)
        y = yd.cpu().numpy().astype(np.complex128)
        tol = 1e-10 if precision == "fp64" else 1e-5
        off = 0
        for (sc, ctx), (_, N, L, nrhs) in zip(ens, ENSEMBLES):
            t = mie.t_diagonal(L, sc.k, sc.radii, sc.n_rel)
            W = translation.coupling_matrix(sc.positions, sc.k, L)
            for r in range(nrhs):
                xs = x[off:off + N * sc.nmax].reshape(N, sc.nmax)
                ref = solve.apply_M(W, t, xs)
                got = y[off:off + N * sc.nmax].reshape(N, sc.nmax)
                assert rel(got, ref) <= tol, (N, L, r)
                off += N * sc.nmax
        assert off == n
    finally:
        B.celes_batch_destroy(b)


@pytest.mark.parametrize("mode,tol,bound", [(B.CELES_SOLVE_MIXED, 1e-6, 1e-5), (B.CELES_SOLVE_FP64, 1e-11, 1e-9)])
def test_batched_solve_matches_dense_lu(batch_setup, mode, tol, bound):
    ens = batch_setup
    refs = _references(ens)
    b = B.celes_batch_create([c for _, c in ens], restart=20)
    try:
        code, infos = B.celes_batch_solve(b, len(ens), tol, mode=mode, restart=20)
        assert code == B.CELES_OK
        for inf in infos:
            assert inf["status"] == B.CELES_OK and inf["residual"] <= tol
        q = 0
        for (sc, ctx), (_, N, L, nrhs) in zip(ens, ENSEMBLES):
            got = B.celes_get_coefficients(ctx)
            for r in range(nrhs):
                assert rel(got[r], refs[q]) <= bound, (N, L, r)
                q += 1
    finally:
        B.celes_batch_destroy(b)


def test_batched_equals_one_by_one(batch_setup):
    ens = batch_setup
    b = B.celes_batch_create([c for _, c in ens], restart=15)
    try:
        B.celes_batch_solve(b, len(ens), 1e-8, mode=B.CELES_SOLVE_FP64, restart=15)
        batched = [B.celes_get_coefficients(c) for _, c in ens]
    finally:
        B.celes_batch_destroy(b)
    for (sc, ctx), got in zip(ens, batched):
        B.celes_solve(ctx, 1e-8, mode=B.CELES_SOLVE_FP64, restart=15, use_precond=False)
        single = B.celes_get_coefficients(ctx)
        assert rel(got, single) <= 1e-6


def test_batch_rejects_bad_use(batch_setup):
    ens = batch_setup
    with pytest.raises(B.CelesError):
        B.celes_batch_create([])
    b = B.celes_batch_create([ens[0][1]])
    try:
        opts = B.celes_solve_opts(B.CELES_SOLVE_MIXED, 20, 100, 4, B.CELES_X0_ZERO, 0, 1e-5, 0)
        info = (B.celes_solve_info * 1)()
        assert B.load().celes_batch_solve(b, 1e-6, opts, info) == B.CELES_EINVAL
    finally:
        B.celes_batch_destroy(b)


def test_batched_solve_ignores_stale_device_memory():
    """Systems that stop their Krylov cycle at different steps leave the later
    basis vectors of their segment unwritten; the update must not read them.
    Device memory full of NaN is freed first, so that the batch's fresh buffers
    are likely to reuse it (a plain first allocation would read as zeros)."""
    junk = torch.full((48 * 1024 * 1024,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    del junk
    torch.cuda.empty_cache()
    ens = []
    try:
        for q, (N, L) in enumerate([(20, 2), (35, 3)]):
            sc = synth.random_cluster(89, 10 + q, N, L, radius=100.0, fill=0.15, n=1.5 + 0.01j)
            ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, L)
            B.celes_set_incident(ctx, [B.make_incident("plane", beta=0.2, alpha=0.1, pol=2)])
            ens.append((sc, ctx))
        b = B.celes_batch_create([c for _, c in ens])
        try:
            code, infos = B.celes_batch_solve(b, len(ens), 1e-8, mode=B.CELES_SOLVE_MIXED)
            assert code == B.CELES_OK
        finally:
            B.celes_batch_destroy(b)
        for sc, ctx in ens:
            L = sc.lmax
            got = B.celes_get_coefficients(ctx)
            assert np.all(np.isfinite(got))
            t = mie.t_diagonal(L, sc.k, sc.radii, sc.n_rel)
            a = incident.plane_wave_coeffs(L, sc.k, sc.positions, 0.2, 0.1, 2)
            assert rel(got[0], solve.solve_dense(sc.positions, sc.k, L, t, a)) <= 1e-6
    finally:
        for _, ctx in ens:
            B.celes_destroy(ctx)
