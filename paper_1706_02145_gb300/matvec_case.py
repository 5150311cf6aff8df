"""Run one synthetic case of a hot-path operation (for timing and profiling).

  python -m paper_1706_02145_gb300.matvec_case --N 6000 --lmax 4 --precision fp32 --kernel rtr --reps 2
  python -m paper_1706_02145_gb300.matvec_case --op precond --N 10000 --edge 900 --precision fp32
  python -m paper_1706_02145_gb300.matvec_case --op batch --ensembles 12 --rhs 4 --precision fp32

--op coupling (default): the coupling matvec y = W x on the bench workload's
  recipe (lognormal radii, cylinder slab at fill 0.3) with N spheres and the
  given lmax, or the 100 000-sphere slab (--recipe large).
--op precond: builds the block-diagonal preconditioner with cuboids of
  --edge nm on the same recipe and applies it.
--op batch: the batched operator (I - T W) over --ensembles ensembles of the
  multi-ensemble recipe (sizes scaled by 0.4) with --rhs plane waves each.
Runs `reps` operations through the C ABI and prints the time of the last one.
"""

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["coupling", "precond", "batch"], default="coupling")
    ap.add_argument("--N", type=int, default=6000)
    ap.add_argument("--lmax", type=int, default=4)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--kernel", choices=["auto", "direct", "rtr"], default="auto")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--recipe", choices=["slab", "large"], default="slab",
                    help="slab: the bench recipe (Gaussian-beam cylinder slab) with N spheres and lmax; "
                         "large: the 100 000-sphere monodisperse slab (lmax 3, N and lmax ignored)")
    ap.add_argument("--edge", type=float, default=900.0, help="preconditioner cuboid edge (nm)")
    ap.add_argument("--ensembles", type=int, default=12)
    ap.add_argument("--rhs", type=int, default=4)
    a = ap.parse_args()
    import torch
    import synth
    from paper_1706_02145_gb300 import binding as B
    B.load()
    prec = B.CELES_FP32 if a.precision == "fp32" else B.CELES_FP64
    dt = torch.complex64 if prec == B.CELES_FP32 else torch.complex128
    g = torch.Generator(device="cuda").manual_seed(0)
    if a.op == "batch":
        scenes = []
        for e in range(a.ensembles):
            scenes.append(synth.config3(e, n_rhs=a.rhs, N=max(80, int(0.4 * synth.config3_size(e)))))
        ctxs = []
        for sc in scenes:
            c = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax)
            B.celes_set_incident(c, [B.make_incident("plane", beta=i.beta, alpha=i.alpha, pol=i.pol)
                                     for i in sc.incidents])
            ctxs.append(c)
        bt = B.celes_batch_create(ctxs)
        n = B.celes_batch_num_unknowns(bt)
        x = torch.randn(n, dtype=dt, device="cuda", generator=g)
        y = torch.empty_like(x)
        t = 0.0
        for _ in range(a.reps):
            t0 = time.perf_counter()
            B.celes_batch_master_matvec(bt, x, y, precision=prec)
            t = time.perf_counter() - t0
        pairs = sum(sc.N * (sc.N - 1) * len(sc.incidents) for sc in scenes)
        print(f"batch of {len(scenes)} ensembles x {a.rhs} RHS, {a.precision}: {t * 1e3:.3f} ms, "
              f"{pairs / t:.3e} couplings/s")
        B.celes_batch_destroy(bt)
        for c in ctxs:
            B.celes_destroy(c)
        return
    kern = {"auto": B.CELES_KERNEL_AUTO, "direct": B.CELES_KERNEL_DIRECT, "rtr": B.CELES_KERNEL_RTR}[a.kernel]
    sc = synth.config2(0, N=a.N, lmax=a.lmax) if a.recipe == "slab" else synth.config5(0)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax, kernel=kern)
    x = torch.randn(sc.N, sc.nmax, dtype=dt, device="cuda", generator=g)
    y = torch.empty_like(x)
    if a.op == "precond":
        B.celes_precond_build(ctx, a.edge)
    t = 0.0
    for _ in range(a.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if a.op == "precond":
            B.celes_precond_apply(ctx, x, y, precision=prec)
        else:
            B.celes_coupling_matvec(ctx, x, y, precision=prec)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    if a.op == "precond":
        print(f"N={sc.N} lmax={sc.lmax} {a.precision} block preconditioner apply (edge {a.edge:g} nm): "
              f"{t * 1e3:.3f} ms")
    else:
        pairs = sc.N * (sc.N - 1)
        print(f"N={sc.N} lmax={sc.lmax} {a.precision} kernel={a.kernel}: {t * 1e3:.3f} ms, {pairs / t:.3e} couplings/s")
    B.celes_destroy(ctx)


if __name__ == "__main__":
    main()
