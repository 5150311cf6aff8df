"""The allocation-free coupling matvec (celes_coupling_matvec_noalloc).

It is meant for callers that cannot call cudaMalloc -- code running under a
host application's own device-memory pool, or latency-critical code that
cannot take the device-wide synchronisation of cudaMalloc/cudaFree -- so it
keeps its scratch in a static device array inside the library.  This test
calls it twice in a row through the C ABI (different inputs, the second call
reusing the array the first one wrote) and compares each result with the
context-based celes_coupling_matvec, within the tolerances of the other GPU
tests.  The file name sorts last so that a stop-at-first-failure run has
already run every other test.
"""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1706_02145_gb300 import binding as B  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    B.load()


def _positions4(sc):
    p4 = np.zeros((sc.N, 4))
    p4[:, :3] = sc.positions
    t = torch.from_numpy(p4).cuda()
    assert t.data_ptr() % 32 == 0
    return t


@pytest.mark.parametrize("precision,tol", [(B.CELES_FP64, 1e-10), (B.CELES_FP32, 1e-5)])
def test_noalloc_matches_context_matvec_on_two_calls(precision, tol):
    dt = torch.complex128 if precision == B.CELES_FP64 else torch.complex64
    cases = [synth.random_cluster(31, 0, 300, 4, radius=100.0, fill=0.25, polydisperse=True),
             synth.random_cluster(31, 1, 157, 3, radius=120.0, fill=0.2)]
    for q, sc in enumerate(cases):
        ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax)
        try:
            x = torch.from_numpy(synth.random_vector(31, 10 + q, (sc.N, sc.nmax))).to(dt).cuda()
            y_ref = torch.zeros_like(x)
            B.celes_coupling_matvec(ctx, x, y_ref, precision=precision)
            pos4 = _positions4(sc)
            y = torch.full_like(x, float("nan"))
            B.celes_coupling_matvec_noalloc(sc.N, sc.lmax, sc.k, pos4, x, y, precision=precision)
            torch.cuda.synchronize()
            a = y.cpu().numpy().astype(np.complex128)
            b = y_ref.cpu().numpy().astype(np.complex128)
            assert np.all(np.isfinite(a))
            assert rel(a, b) < tol
        finally:
            B.celes_destroy(ctx)


def test_noalloc_matches_the_oracle_rows():
    """The allocation-free path against the oracle's on-the-fly FP64 coupling
    rows (Sec. 2.2), not only against the context path it shares kernels
    with."""
    from oracle import translation
    sc = synth.random_cluster(31, 3, 120, 4, radius=100.0, fill=0.25, polydisperse=True)
    x_np = synth.random_vector(31, 20, (sc.N, sc.nmax))
    rows = [0, 1, 17, 58, 99, sc.N - 1]
    ref = translation.coupling_matvec_rows(sc.positions, sc.k, sc.lmax, x_np, rows)
    pos4 = _positions4(sc)
    for precision, dt, tol in [(B.CELES_FP64, torch.complex128, 1e-10), (B.CELES_FP32, torch.complex64, 1e-5)]:
        x = torch.from_numpy(x_np).to(dt).cuda()
        for _ in range(2):  # the second call reuses the scratch the first one wrote
            y = torch.full_like(x, float("nan"))
            B.celes_coupling_matvec_noalloc(sc.N, sc.lmax, sc.k, pos4, x, y, precision=precision)
            torch.cuda.synchronize()
            got = y.cpu().numpy().astype(np.complex128)[rows]
            assert rel(got, ref) < tol


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # N * nmax * 16 bytes above 32 MiB is refused before any GPU work.  The
    # buffers are allocated at the full size anyway (about 38 MB each), so
    # that a regression of the size check computes on valid memory and fails
    # the assertion instead of touching memory out of bounds.
    N, L = 50_000, 4
    nmax = 2 * L * (L + 2)
    g = np.arange(N)
    p4 = np.zeros((N, 4))
    p4[:, 0], p4[:, 1], p4[:, 2] = 400.0 * (g % 40), 400.0 * ((g // 40) % 40), 400.0 * (g // 1600)
    pos4 = torch.from_numpy(p4).cuda()
    x = torch.zeros((N, nmax), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    k = 2 * np.pi / 550.0
    code = B.celes_coupling_matvec_noalloc(N, L, k, pos4, x, y, precision=B.CELES_FP64, check=False)
    assert code == B.CELES_ETOOBIG
    code = B.celes_coupling_matvec_noalloc(N, L, k, pos4, x, x, precision=B.CELES_FP64, check=False)
    assert code in (B.CELES_ETOOBIG, B.CELES_EINVAL)
    n_small = 1000
    code = B.celes_coupling_matvec_noalloc(n_small, L, k, pos4, x, x, precision=B.CELES_FP64, check=False)
    assert code == B.CELES_EINVAL  # x and y alias
