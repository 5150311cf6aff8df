"""Reflected / transmitted power (App. D) on the GPU against the oracle with
the same solution coefficients and the same quadrature (1e-10 relative), and
energy conservation R + T = 1 for lossless spheres solved to 1e-12 (1e-8)."""

import numpy as np
import pytest

import synth
from oracle import power

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1706_02145_gb300 import binding as B  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    B.load()


@pytest.mark.parametrize("n,L,N", [(1.6 + 0j, 3, 6), (1.5 + 0.05j, 2, 12)])
def test_power_matches_oracle_and_conserves_energy(n, L, N):
    sc = synth.random_cluster(73, N, N, L, radius=110.0, fill=0.12, n=n)
    w, focus, aG = 1200.0, (30.0, -20.0, 0.0), -np.pi / 2
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, L)
    try:
        B.celes_set_incident(ctx, [B.make_incident("gaussian", waist=w, focus=focus, alpha_G=aG, n_beta=256,
                                                   E0=0.7 + 0.2j)])
        B.celes_solve(ctx, 1e-12, mode=B.CELES_SOLVE_FP64)
        b = B.celes_get_coefficients(ctx)[0]
        R, T = B.celes_power(ctx, n_beta=96, n_alpha=96)
        Ro, To = power.reflect_transmit(L, sc.k, sc.positions, b, w, focus, aG, E0=0.7 + 0.2j, n_beta=96, n_alpha=96)
        assert abs(R - Ro) <= 1e-10 * Ro and abs(T - To) <= 1e-10 * To
        if n.imag == 0.0:
            assert abs(R + T - 1.0) < 1e-8
        else:
            assert R + T < 1.0 - 1e-4
    finally:
        B.celes_destroy(ctx)


def test_power_needs_a_gaussian_beam():
    sc = synth.random_cluster(73, 1, 4, 2, radius=110.0, fill=0.12)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, 2)
    try:
        B.celes_set_incident(ctx, [B.make_incident("plane")])
        B.celes_solve(ctx, 1e-8, mode=B.CELES_SOLVE_FP64)
        with pytest.raises(B.CelesError):
            B.celes_power(ctx)
    finally:
        B.celes_destroy(ctx)


def test_s11_matches_oracle():
    from oracle import farfield
    sc = synth.random_cluster(73, 5, 10, 3, radius=110.0, fill=0.15, n=1.5 + 0.01j)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, 3)
    try:
        B.celes_set_incident(ctx, [B.make_incident("plane", pol=1), B.make_incident("plane", pol=2)])
        B.celes_solve(ctx, 1e-12, mode=B.CELES_SOLVE_FP64)
        b = B.celes_get_coefficients(ctx)
        betas = np.linspace(0.0, np.pi, 19)
        got = B.celes_s11(ctx, betas, 0, 1, n_alpha=24)
        ref = farfield.s11_azimuthal(3, sc.k, sc.positions, b[0], b[1], betas, n_alpha=24)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-10
    finally:
        B.celes_destroy(ctx)
