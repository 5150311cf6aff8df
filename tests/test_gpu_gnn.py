"""Learned initial guess (graph network over 16 nearest neighbours).

1. The hand-written forward and backward kernels (tcgen05 BF16 GEMMs, FP32
   accumulation) against a PyTorch autograd reference of the same network on
   the CPU, with the GEMM operands rounded to BF16 as the kernels do:
   loss to 1e-3 relative, every parameter gradient to 3e-2 relative L2 (the
   backward GEMMs round their operands to BF16 as well).
2. Training on solved ensembles lowers the loss; a solve started from the
   learned guess still reaches the FP64 residual tolerance and the oracle
   solution (the residual decides; the solver falls back to T a).
"""

import numpy as np
import pytest

import synth
from oracle import incident, mie, solve

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


def _solved(seed, N, L, beta=0.0):
    sc = synth.random_cluster(41, seed, N, L, radius=100.0, fill=0.25, n=1.55 + 0.01j)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, L)
    B.celes_set_incident(ctx, [B.make_incident("plane", beta=beta, alpha=0.3, pol=2)])
    B.celes_solve(ctx, 1e-10, mode=B.CELES_SOLVE_FP64)
    return sc, ctx


def _bf(x):
    return x.to(torch.bfloat16).to(torch.float32)


def _reference(sc, ctx, params, W, layers, L):
    nmax = sc.nmax
    F = (2 * nmax + 3 + 7) // 8 * 8
    OUTP = (2 * nmax + 7) // 8 * 8
    KN = 16
    ta = (B.celes_get_tmatrix(ctx) * B.celes_get_incident_coefficients(ctx)[0])
    b = B.celes_get_coefficients(ctx)[0]
    ta_r = np.stack([ta.real, ta.imag], axis=-1).reshape(sc.N, 2 * nmax)
    b_r = np.stack([b.real, b.imag], axis=-1).reshape(sc.N, 2 * nmax)
    scale = 1.0 / np.sqrt(np.mean(ta_r ** 2))
    feat = np.zeros((sc.N, F))
    feat[:, :2 * nmax] = ta_r * scale
    feat[:, 2 * nmax] = sc.k * sc.radii
    feat[:, 2 * nmax + 1] = sc.n_rel.real - 1.0
    feat[:, 2 * nmax + 2] = sc.n_rel.imag
    pos = sc.positions
    d = pos[None, :, :].astype(np.float32) - pos[:, None, :].astype(np.float32)
    dist = np.sum(d * d, axis=2)
    np.fill_diagonal(dist, np.inf)
    nbr = np.argsort(dist, axis=1, kind="stable")[:, :KN]
    rel = pos[nbr] - pos[:, None, :]
    dd = np.linalg.norm(rel, axis=2)
    s = sc.k / (2 * np.pi)
    ef = np.zeros((sc.N, KN, 8))
    ef[:, :, :3] = rel * s
    ef[:, :, 3] = dd * s
    ef[:, :, 4] = 1.0 / (sc.k * dd)
    tgt = np.zeros((sc.N, OUTP))
    tgt[:, :2 * nmax] = (b_r - ta_r) * scale
    # parameters in export order
    shapes = [(W, F)] + [(W, 2 * W + 8), (W, 2 * W)] * layers + [(OUTP, W)]
    ts, off = [], 0
    for (o, i) in shapes:
        w = torch.tensor(params[off:off + o * i].reshape(o, i), requires_grad=True)
        off += o * i
        bb = torch.tensor(params[off:off + o], requires_grad=True)
        off += o
        ts.append((w, bb))
    X = torch.tensor(feat, dtype=torch.float32)
    nb = torch.tensor(nbr)
    E = torch.tensor(ef, dtype=torch.float32)
    h = torch.relu(_bf(X) @ _bf(ts[0][0]).T + ts[0][1])
    for l in range(layers):
        wm, bm = ts[1 + 2 * l]
        wu, bu = ts[2 + 2 * l]
        xe = torch.cat([h[nb], h[:, None, :].expand(-1, KN, -1), E], dim=2)
        m = torch.relu(_bf(xe) @ _bf(wm).T + bm)
        agg = m.mean(dim=1)
        u = torch.cat([h, agg], dim=1)
        h = h + torch.relu(_bf(u) @ _bf(wu).T + bu)
    o = _bf(h) @ _bf(ts[-1][0]).T + ts[-1][1]
    loss = torch.mean((o - torch.tensor(tgt, dtype=torch.float32)) ** 2)
    loss.backward()
    grads = np.concatenate([np.concatenate([w.grad.numpy().ravel(), bb.grad.numpy()]) for (w, bb) in ts])
    return float(loss.detach()), grads, shapes


def test_gnn_forward_and_backward_match_autograd():
    L, W, layers = 2, 32, 2
    sc, ctx = _solved(0, 140, L)
    g = B.celes_gnn_create(L, width=W, layers=layers, seed=3)
    try:
        B.celes_gnn_train(g, ctx, steps=1, lr=1e-2)    # makes the zero-initialised output layer nonzero
        params = B.celes_gnn_export(g, 0)
        loss = B.celes_gnn_train(g, ctx, steps=0)      # loss and gradients only
        grads = B.celes_gnn_export(g, 1)
        ref_loss, ref_grads, shapes = _reference(sc, ctx, params, W, layers, L)
        assert abs(loss - ref_loss) <= 1e-3 * abs(ref_loss)
        off = 0
        for (o, i) in shapes:
            n = o * i + o
            a, r = grads[off:off + n], ref_grads[off:off + n]
            assert np.linalg.norm(a - r) <= 3e-2 * np.linalg.norm(r) + 1e-12, (o, i)
            off += n
    finally:
        B.celes_gnn_destroy(g)
        B.celes_destroy(ctx)


def test_gnn_training_and_learned_guess_solve():
    L = 2
    g = B.celes_gnn_create(L, width=64, layers=3, seed=5)
    train = [_solved(s, 160, L, beta=0.1 * s) for s in range(1, 5)]
    try:
        first = [B.celes_gnn_train(g, ctx, steps=1, lr=2e-3) for _, ctx in train]
        for _ in range(40):
            for _, ctx in train:
                B.celes_gnn_train(g, ctx, steps=1, lr=2e-3)
        last = [B.celes_gnn_train(g, ctx, steps=0) for _, ctx in train]
        assert np.mean(last) < 0.7 * np.mean(first)
        # held-out ensemble: learned first iterate, the FP64 residual decides
        sc = synth.random_cluster(41, 99, 160, L, radius=100.0, fill=0.25, n=1.55 + 0.01j)
        ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, L)
        try:
            B.celes_set_incident(ctx, [B.make_incident("plane", beta=0.25, alpha=0.3, pol=2)])
            B.celes_gnn_predict(g, ctx)
            info = B.celes_solve(ctx, 1e-6, mode=B.CELES_SOLVE_MIXED, x0=B.CELES_X0_LEARNED)
            assert info["residual"] <= 1e-6 and info["guess_used"] in (0, 1)
            b = B.celes_get_coefficients(ctx)[0]
            t = mie.t_diagonal(L, sc.k, sc.radii, sc.n_rel)
            a = incident.plane_wave_coeffs(L, sc.k, sc.positions, 0.25, 0.3, 2)
            ref = solve.solve_dense(sc.positions, sc.k, L, t, a)
            assert np.linalg.norm(b - ref) <= 1e-5 * np.linalg.norm(ref)
        finally:
            B.celes_destroy(ctx)
    finally:
        B.celes_gnn_destroy(g)
        for _, ctx in train:
            B.celes_destroy(ctx)


def test_gnn_at_the_learned_guess_shape_matches_autograd():
    # width 128, 3 message-passing layers, lmax 3 (the stated network)
    L, W, layers = 3, 128, 3
    sc, ctx = _solved(7, 150, L)
    g = B.celes_gnn_create(L, width=W, layers=layers, seed=11)
    try:
        B.celes_gnn_train(g, ctx, steps=1, lr=1e-2)
        params = B.celes_gnn_export(g, 0)
        loss = B.celes_gnn_train(g, ctx, steps=0)
        grads = B.celes_gnn_export(g, 1)
        ref_loss, ref_grads, shapes = _reference(sc, ctx, params, W, layers, L)
        assert abs(loss - ref_loss) <= 1e-3 * abs(ref_loss)
        off = 0
        for (o, i) in shapes:
            n = o * i + o
            a, r = grads[off:off + n], ref_grads[off:off + n]
            assert np.linalg.norm(a - r) <= 3e-2 * np.linalg.norm(r) + 1e-12, (o, i)
            off += n
    finally:
        B.celes_gnn_destroy(g)
        B.celes_destroy(ctx)


def test_gnn_stored_examples_train_like_their_contexts():
    # an example stored from a context and then trained without it gives the
    # same losses and parameters as training on the context itself
    L = 2
    sc, ctx = _solved(3, 120, L)
    g1 = B.celes_gnn_create(L, width=32, layers=2, seed=9)
    g2 = B.celes_gnn_create(L, width=32, layers=2, seed=9)
    try:
        idx = B.celes_gnn_add_example(g2, ctx)
        assert idx == 0 and B.celes_gnn_num_examples(g2) == 1
        B.celes_destroy(ctx)
        ctx = None
        sc2, ctx2 = _solved(3, 120, L)
        try:
            l1 = [B.celes_gnn_train(g1, ctx2, steps=1, lr=3e-3) for _ in range(5)]
        finally:
            B.celes_destroy(ctx2)
        l2 = [B.celes_gnn_train_example(g2, idx, steps=1, lr=3e-3) for _ in range(5)]
        assert np.allclose(l1, l2, rtol=1e-5, atol=0)
        # (the feature scale is a sum reduced with atomics: equal to rounding)
        p1, p2 = B.celes_gnn_export(g1, 0), B.celes_gnn_export(g2, 0)
        assert np.linalg.norm(p1 - p2) <= 1e-5 * np.linalg.norm(p1)
        B.celes_gnn_clear_examples(g2)
        assert B.celes_gnn_num_examples(g2) == 0
        with pytest.raises(B.CelesError):
            B.celes_gnn_train_example(g2, 0)
    finally:
        B.celes_gnn_destroy(g1)
        B.celes_gnn_destroy(g2)
        if ctx is not None:
            B.celes_destroy(ctx)
