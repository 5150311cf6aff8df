"""Run coupling matvecs of one synthetic case (for timing and profiling).

  python -m paper_1706_02145_gb300.matvec_case --N 6000 --lmax 4 --precision fp32 --kernel rtr --reps 2

Builds the packing of the bench workload's recipe (lognormal radii, cylinder
slab at fill 0.3) with N spheres and the given lmax, or the 100 000-sphere
slab (`--recipe large`), runs `reps` coupling matvecs through the C ABI and
prints the time of the last one.
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
    ap.add_argument("--N", type=int, default=6000)
    ap.add_argument("--lmax", type=int, default=4)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--kernel", choices=["auto", "direct", "rtr"], default="auto")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--recipe", choices=["slab", "large"], default="slab",
                    help="slab: the bench recipe (Gaussian-beam cylinder slab) with N spheres and lmax; "
                         "large: the 100 000-sphere monodisperse slab (lmax 3, N and lmax ignored)")
    a = ap.parse_args()
    import torch
    import synth
    from paper_1706_02145_gb300 import binding as B
    B.load()
    kern = {"auto": B.CELES_KERNEL_AUTO, "direct": B.CELES_KERNEL_DIRECT, "rtr": B.CELES_KERNEL_RTR}[a.kernel]
    prec = B.CELES_FP32 if a.precision == "fp32" else B.CELES_FP64
    sc = synth.config2(0, N=a.N, lmax=a.lmax) if a.recipe == "slab" else synth.config5(0)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax, kernel=kern)
    dt = torch.complex64 if prec == B.CELES_FP32 else torch.complex128
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(sc.N, sc.nmax, dtype=dt, device="cuda", generator=g)
    y = torch.empty_like(x)
    t = 0.0
    for _ in range(a.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.celes_coupling_matvec(ctx, x, y, precision=prec)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    pairs = sc.N * (sc.N - 1)
    print(f"N={sc.N} lmax={sc.lmax} {a.precision} kernel={a.kernel}: {t * 1e3:.3f} ms, {pairs / t:.3e} couplings/s")
    B.celes_destroy(ctx)


if __name__ == "__main__":
    main()
