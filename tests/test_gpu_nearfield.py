"""Near field (Sec. 2.1): scattered field from the GPU solution's expansion
coefficients, incident plane wave and Gaussian beam, against the oracle's
SVWF sums and PVWF / angular-spectrum evaluations (FP64: 1e-10 scattered,
1e-12 plane wave, 1e-9 Gaussian beam, which the two sides integrate with
different quadratures of the same integral); points inside a sphere are NaN."""

import numpy as np
import pytest

import synth
from oracle import incident, svwf

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


def _grid(sc, n=9):
    lo = sc.positions.min(axis=0) - 300.0
    hi = sc.positions.max(axis=0) + 300.0
    g = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(lo[0] + g * (hi[0] - lo[0]), lo[1] + g * (hi[1] - lo[1]), indexing="ij")
    z = 0.5 * (lo[2] + hi[2])
    pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)
    # plus the centre of sphere 0 (inside) and a point just outside sphere 1
    d = np.array([0.0, 0.0, 1.0])
    extra = [sc.positions[0], sc.positions[1] + (sc.radii[1] * 1.01) * d]
    return np.concatenate([pts, np.array(extra)], axis=0)


def _inside(sc, pts):
    d = np.linalg.norm(pts[:, None, :] - sc.positions[None, :, :], axis=2)
    return np.any(d < sc.radii[None, :], axis=1)


@pytest.mark.parametrize("L", [2, 4])
def test_scattered_and_plane_wave_field(L):
    sc = synth.random_cluster(53, L, 8, L, radius=120.0, fill=0.15, n=1.6 + 0.05j, polydisperse=True)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, L)
    try:
        B.celes_set_incident(ctx, [B.make_incident("plane", beta=0.3, alpha=0.8, pol=1, E0=1.0)])
        with pytest.raises(B.CelesError):
            B.celes_nearfield(ctx, np.zeros((1, 3)) + 1e5, what=0)  # no solution yet
        B.celes_solve(ctx, 1e-12, mode=B.CELES_SOLVE_FP64)
        b = B.celes_get_coefficients(ctx)[0]
        pts = _grid(sc)
        ins = _inside(sc, pts)
        assert ins.any() and (~ins).sum() > 50
        Es = B.celes_nearfield(ctx, pts, what=0)
        Ei = B.celes_nearfield(ctx, pts, what=1)
        Et = B.celes_nearfield(ctx, pts, what=2)
        assert np.all(np.isnan(Es[ins])) and np.all(np.isnan(Et[ins]))
        out = pts[~ins]
        ref_s = np.zeros((out.shape[0], 3), dtype=complex)
        for i in range(sc.N):
            ref_s += svwf.field_expansion(3, b[i], L, sc.k, out, origin=sc.positions[i])
        ref_i = svwf.pvwf(1, 0.8, 0.3, sc.k, pts)
        assert rel(Es[~ins], ref_s) <= 1e-10
        assert rel(Ei, ref_i) <= 1e-12
        assert rel(Et[~ins], ref_s + ref_i[~ins]) <= 1e-10
    finally:
        B.celes_destroy(ctx)


def test_gaussian_beam_field():
    sc = synth.random_cluster(53, 7, 5, 2, radius=120.0, fill=0.1)
    w, focus, aG = 1500.0, (100.0, -50.0, 200.0), -np.pi / 2
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, 2)
    try:
        B.celes_set_incident(ctx, [B.make_incident("gaussian", waist=w, focus=focus, alpha_G=aG, n_beta=128)])
        g = np.linspace(-1500.0, 1500.0, 7)
        pts = np.array([[x, y, z] for x in g for y in g[::2] for z in (-400.0, 300.0)])
        E = B.celes_nearfield(ctx, pts, what=1)
        ref = incident.gaussian_beam_field(sc.k, w, focus, aG, pts, n_beta=256, n_alpha=256)
        assert rel(E, ref) <= 1e-9
    finally:
        B.celes_destroy(ctx)
