#!/usr/bin/env python
"""Benchmark of the multi-sphere T-matrix hot path on GB300.

Workload: 10 000 polydisperse spheres (lognormal radii, mean 150 nm, sigma of
ln R 0.1), n = 1.5 + 0.001i, lambda = 550 nm, lmax = 4 (48 coefficients per
sphere), random packing at fill 0.3 in a 2 um thick cylindrical slab, Gaussian
beam of waist 2 um (synthetic, seeded; see synth/).

One step = one pass of the path over the resident inputs:
  incident coefficients + T a (Gaussian-beam beta quadrature)
  -> mixed-precision solve to relative residual 1e-6 (FP32 coupling matvecs in
     GMRES, FP64 coupling matvecs for the refinement residuals)
  -> far-field amplitudes on a 32 x 64 direction grid.

metric: sphere-pair couplings/s = (coupling matvecs in the step) * N (N - 1)
divided by the step time; plus the time to 1e-6 of the chosen form against the
plain FP64 GMRES solve on the same GPU and inputs.

Outside the timed steps the same context is solved again to relative
residual 1e-10 (FP64 refinement); the oracle's FP64 residual on sampled
receiver rows (cpu_baseline leg) certifies that reference, and every solve in
the line reports its coefficient error against it (error_vs_fp64_oracle).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --case coupling|precond|batch [...]   (one operation, for profiling)

Multi-GPU: replicas (each rank solves its own copy; no data exchange), launched
by torchrun; value = all ranks' couplings / max-over-ranks time.
"""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time
from functools import partial

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sphere-pair couplings/s; time to 1e-6 residual, chosen form vs plain FP64"
UNIT = "sphere-pair couplings/s"
TOL = 1e-6
REF_TOL = 1e-10           # the certified reference solve


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=10_000, help="spheres (default: the full workload)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 time-to-1e-6 run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-rows", type=int, default=0, help="receivers in the CPU sample (0 = auto)")
    ap.add_argument("--small-n", type=int, default=2000, help="spheres of the measured plain-FP64 comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched multi-ensemble measurement")
    ap.add_argument("--batched-ensembles", type=int, default=64)
    ap.add_argument("--batched-rhs", type=int, default=8)
    ap.add_argument("--batched-restart", type=int, default=100, help="GMRES restart of both batched forms")
    ap.add_argument("--batched-scale", type=float, default=1.0,
                    help="sphere counts of the multi-ensemble workload times this factor (1 = as stated)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-initial-guess measurement")
    ap.add_argument("--no-precond", action="store_true", help="skip the block-preconditioned solve")
    ap.add_argument("--no-certify", action="store_true",
                    help="skip the 1e-10 reference solve and the oracle residual on sampled rows")
    ap.add_argument("--plain-full", action="store_true",
                    help="also run the full-size plain FP64 GMRES solve to 1e-6 uncapped (about 10 min)")
    ap.add_argument("--learned-c4", action="store_true",
                    help="run only the learned-guess workload at its stated size (training and 100 evaluations)")
    ap.add_argument("--c4-train", type=int, default=2000, help="--learned-c4: training ensembles")
    ap.add_argument("--c4-eval", type=int, default=100, help="--learned-c4: evaluation ensembles (8000 spheres)")
    ap.add_argument("--c4-epochs", type=int, default=20, help="--learned-c4: training epochs")
    ap.add_argument("--c5", action="store_true",
                    help="run only the 100 000-sphere workload end to end (preconditioned mixed solve to 1e-6)")
    ap.add_argument("--c5-edge", type=float, default=1000.0, help="--c5: preconditioner cuboid edge (nm)")
    ap.add_argument("--plain-full-only", action="store_true",
                    help="run only the uncapped plain FP64 solve of the bench workload beside the chosen form")
    ap.add_argument("--inner-tol", type=str, default="1e-5",
                    help="--case solve: comma-separated inner tolerances of the mixed solve to compare")
    ap.add_argument("--case", choices=["coupling", "precond", "batch", "solve"], default=None,
                    help="run one operation on a synthetic case and print its time (profiling); see run_case")
    ap.add_argument("--lmax", type=int, default=4, help="--case: degree")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32", help="--case: precision")
    ap.add_argument("--kernel", choices=["auto", "direct", "rtr"], default="auto", help="--case: coupling kernel")
    ap.add_argument("--reps", type=int, default=2, help="--case: repetitions (time of the last printed)")
    ap.add_argument("--recipe", choices=["slab", "large"], default="slab",
                    help="--case: slab = the bench recipe with --N spheres and --lmax; large = the 100 000-sphere "
                         "monodisperse slab (lmax 3)")
    ap.add_argument("--edge", type=float, default=900.0, help="--case precond: cuboid edge (nm)")
    ap.add_argument("--autotune", type=int, default=1, help="--case coupling: 1 = tune the launch shape, 0 = built-in")
    ap.add_argument("--variant", type=int, default=-1,
                    help="--case coupling: force the FP32 launch shape (0-7: bit 0 the alternative shape, bit 1 the "
                         "cluster reduction, bit 2 the reduction in L2)")
    ap.add_argument("--chunks", type=int, default=0, help="--case coupling: source chunks (0: automatic)")
    ap.add_argument("--ensembles", type=int, default=12, help="--case batch: ensembles")
    ap.add_argument("--rhs", type=int, default=0,
                    help="--case: right-hand sides (0 = 1 for coupling, 4 plane waves per ensemble for batch)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def flops_per_pair(lmax):
    """Algorithmic flops per ordered sphere pair and RHS of the coupling kernel
    the library runs (rotation-translation-rotation), counted by the library
    from its own compile-time tables (celes_flops_per_pair)."""
    from paper_1706_02145_gb300 import binding as B
    return B.celes_flops_per_pair(lmax, B.CELES_KERNEL_AUTO)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("coupling_kernel.cuh", "coupling_tables.cuh", "coupling_launch.cuh", "rtr_kernel.cuh",
              "rtr_tables.cuh"):
        with open(os.path.join(ROOT, "paper_1706_02145_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key, shape=None):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or
    None when it is absent, was taken on other kernel source, or holds no
    capture of the launch shape (variant, chunks) `shape`."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(kernel_key)
        if not e or e.get("source_hash") != kernel_source_hash():
            return None
        if "shapes" in e:
            if shape is None:
                return None
            return e["shapes"].get(f"{shape[0]},{shape[1]}", {}).get("dram_bytes_per_launch")
        if shape is None or (e.get("variant"), e.get("chunks")) == tuple(shape):
            return e.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


def cpu_oracle_rate(scene, rows, n_workers, pool=None):
    """Oracle on-the-fly coupling rows on the host cores: (pairs/s, seconds).
    With `pool` (a spawn-context pool) the workers are reused."""
    import multiprocessing as mp
    from oracle import translation  # noqa: F401  (import check before spawning)
    x = np.random.default_rng(1).normal(size=(scene.N, scene.nmax)) * (1 + 0j)
    chunks = [list(rows[q::n_workers]) for q in range(n_workers)]
    chunks = [c for c in chunks if c]
    args = [(scene.positions, scene.k, scene.lmax, x, c) for c in chunks]
    if pool is None:
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(len(chunks)) as p:
            p.starmap(_oracle_rows, args)
        dt = time.perf_counter() - t0
    else:
        t0 = time.perf_counter()
        pool.starmap(_oracle_rows, args)
        dt = time.perf_counter() - t0
    return len(rows) * (scene.N - 1) / dt, dt


def _oracle_rows(pos, k, lmax, x, rows):
    from oracle import translation
    translation.coupling_matvec_rows(pos, k, lmax, x, rows)
    return len(rows)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle as it stands
# ---------------------------------------------------------------------------

def workload_config(N, L, world):
    """The `config` object of both arms' JSON lines."""
    return {"workload": f"Gaussian-beam slab: {N} polydisperse spheres (lognormal R, mean 150 nm), lmax {L}, "
                        "n=1.5+0.001i, lambda 550 nm, cylinder slab fill 0.3, Gaussian beam w=2um; "
                        "step = incident coefficients + FP32/FP64-refined GMRES to 1e-6 + far field",
            "N": N, "lmax": L, "tol": TOL, "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "flushed between steps (256 MB write); inputs resident in HBM"}


def run_reference(args, rank):
    if rank != 0:
        return
    import synth
    scene = synth.config2(0, N=args.N)
    cores = host_cores()
    rows_per_step = args.cpu_rows or 4 * max(cores, 2)
    rng = np.random.default_rng(7)
    import multiprocessing as mp
    times, pairs = [], 0
    with mp.get_context("spawn").Pool(cores) as pool:  # workers started once, outside the timed steps
        for _ in range(max(1, args.warmup)):
            cpu_oracle_rate(scene, list(rng.choice(scene.N, min(cores, scene.N), replace=False)), cores, pool)
        for _ in range(args.steps):
            rows = list(rng.choice(scene.N, rows_per_step, replace=False))
            rate, dt = cpu_oracle_rate(scene, rows, cores, pool)
            times.append(dt)
            pairs += len(rows) * (scene.N - 1)
    value = pairs / sum(times)
    sample = (f"{rows_per_step} receiver rows x {scene.N - 1} sources per step of the oracle's on-the-fly FP64 "
              f"coupling rows (numpy), {cores} spawn workers started once before the timed steps")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(scene.N, scene.lmax, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def _pack_config3(index, n_rhs, scale):
    """Worker: one multi-ensemble scene (spawn pool)."""
    import synth
    N = None if scale >= 1.0 else max(80, int(scale * synth.config3_size(index)))
    return synth.config3(index, n_rhs=n_rhs, N=N)


def run_batched(args, local_rank):
    """The multi-ensemble workload as stated: 64 ensembles (N ~ U[200, 3000],
    lmax 2..5, lambda, R, n and fill drawn per ensemble) with 8 plane waves
    each, solved in one lockstep batched solve (one persistent coupling launch
    per lmax and precision for all 512 systems, the operator replayed from a
    CUDA graph), against the same systems solved one context at a time.
    Packings come from spawn workers on the host cores."""
    import multiprocessing as mp
    import torch
    from paper_1706_02145_gb300 import binding as B
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(max(1, host_cores())) as pool:
        scenes = pool.starmap(_pack_config3, [(e, args.batched_rhs, args.batched_scale)
                                              for e in range(args.batched_ensembles)])
    t_pack = time.perf_counter() - t0
    ctxs = []
    try:
        for sc in scenes:
            c = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax, device=local_rank)
            ctxs.append(c)
            B.celes_set_incident(c, [B.make_incident("plane", beta=i.beta, alpha=i.alpha, pol=i.pol)
                                     for i in sc.incidents])
        bt = B.celes_batch_create(ctxs, restart=args.batched_restart)
        try:
            n = B.celes_batch_num_unknowns(bt)
            x = torch.ones(n, dtype=torch.complex64, device=f"cuda:{local_rank}")
            y = torch.empty_like(x)
            B.celes_batch_master_matvec(bt, x, y, precision=B.CELES_FP32)  # graph capture, warm-up
            reps = 3
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                B.celes_batch_master_matvec(bt, x, y, precision=B.CELES_FP32)
            torch.cuda.synchronize()
            t_mv = (time.perf_counter() - t0) / reps
            pairs = sum(sc.N * (sc.N - 1) * len(sc.incidents) for sc in scenes)
            code, infos = B.celes_batch_solve(bt, len(ctxs), TOL, mode=B.CELES_SOLVE_MIXED,
                                              restart=args.batched_restart, max_iter=20000,
                                              raise_on_noconv=False)
            t_batch = max(i["seconds"] for i in infos)
            res_batch = max(i["residual"] for i in infos)
            its_batch = max(i["iterations"] for i in infos)
            b_batch = [B.celes_get_coefficients(c) for c in ctxs]
        finally:
            B.celes_batch_destroy(bt)
        t_one, res_one, err = 0.0, 0.0, 0.0
        for c, bb in zip(ctxs, b_batch):
            # the iteration budget of celes_solve covers all RHS of the context
            info = B.celes_solve(c, TOL, mode=B.CELES_SOLVE_MIXED, restart=args.batched_restart, use_precond=False,
                                 max_iter=20000 * args.batched_rhs, raise_on_noconv=False)
            t_one += info["seconds"]
            res_one = max(res_one, info["residual"])
            b1 = B.celes_get_coefficients(c)
            err = max(err, float(np.linalg.norm(bb - b1) / np.linalg.norm(b1)))
        return {"ensembles": len(scenes), "rhs_each": args.batched_rhs, "systems": len(scenes) * args.batched_rhs,
                "size_scale": args.batched_scale, "pack_s": t_pack,
                "N_range": [min(sc.N for sc in scenes), max(sc.N for sc in scenes)],
                "spheres_total": int(sum(sc.N for sc in scenes)),
                "lmax_counts": {str(L): sum(1 for sc in scenes if sc.lmax == L) for L in range(1, 6)},
                "operator_fp32_ms": t_mv * 1e3, "operator_couplings_per_s": pairs / t_mv,
                "batched_solve_s": t_batch, "batched_max_iterations": its_batch, "batched_max_residual": res_batch,
                "one_by_one_solve_s": t_one, "one_by_one_max_residual": res_one, "speedup": t_one / t_batch,
                "batched_vs_one_by_one_max_rel_l2": err,
                "restart": args.batched_restart,
                "note": "mixed FP32/FP64 restarted GMRES to 1e-6, no preconditioner, first iterate T a, both forms"}
    finally:
        for c in ctxs:
            B.celes_destroy(c)


def run_learned(args, local_rank):
    """The graph-network first iterate: trained on solved ensembles of the
    learned-guess recipe (R = 100 nm, n = 1.52, L = 3, plane wave, fill 0.25;
    N reduced to 800..1600 so the measurement takes seconds), evaluated on a
    held-out ensemble of 3000 spheres against the T a start (mixed solve to
    1e-6)."""
    import synth
    from paper_1706_02145_gb300 import binding as B
    train = []
    try:
        t0 = time.perf_counter()
        for i in range(6):
            sc = synth.config4(i, N=800 + 160 * i, fill=0.25)
            c = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax, device=local_rank)
            train.append(c)
            B.celes_set_incident(c, [B.make_incident("plane", beta=0.0, alpha=0.0, pol=2)])
            B.celes_solve(c, 1e-8, mode=B.CELES_SOLVE_MIXED)
        t_solve = time.perf_counter() - t0
        g = B.celes_gnn_create(3, width=128, layers=3, seed=1, device=local_rank)
        try:
            t0 = time.perf_counter()
            first = float(np.mean([B.celes_gnn_train(g, c, steps=0) for c in train]))
            epochs = 60
            for _ in range(epochs):
                for c in train:
                    B.celes_gnn_train(g, c, steps=1, lr=1e-3)
            last = float(np.mean([B.celes_gnn_train(g, c, steps=0) for c in train]))
            t_train = time.perf_counter() - t0
            ev = synth.config4(1000, N=3000, fill=0.25)
            ce = B.celes_create(ev.positions, ev.radii, ev.n_sphere, ev.n0, ev.k0, ev.lmax, device=local_rank)
            try:
                B.celes_set_incident(ce, [B.make_incident("plane", beta=0.0, alpha=0.0, pol=2)])
                B.celes_solve(ce, TOL, mode=B.CELES_SOLVE_MIXED)  # warm-up
                base = B.celes_solve(ce, TOL, mode=B.CELES_SOLVE_MIXED)
                t0 = time.perf_counter()
                B.celes_gnn_predict(g, ce)
                t_pred = time.perf_counter() - t0
                lg = B.celes_solve(ce, TOL, mode=B.CELES_SOLVE_MIXED, x0=B.CELES_X0_LEARNED)
            finally:
                B.celes_destroy(ce)
        finally:
            B.celes_gnn_destroy(g)
        return {"train_ensembles": len(train), "train_N": [800 + 160 * i for i in range(6)], "epochs": epochs,
                "train_solve_s": t_solve, "train_s": t_train, "loss_first": first, "loss_last": last,
                "eval_N": 3000, "ta_iterations": base["iterations"], "ta_s": base["seconds"],
                "learned_iterations": lg["iterations"], "learned_s": lg["seconds"], "predict_s": t_pred,
                "learned_guess_used": lg["guess_used"], "learned_residual": lg["residual"]}
    finally:
        for c in train:
            B.celes_destroy(c)


def _pack_config4(index, N=None):
    """Worker: one learned-guess ensemble (positions, radii, n) by its seed."""
    import synth
    sc = synth.config4(index, N=N)
    return index, sc.positions, sc.radii, sc.n_sphere, sc.name


def run_learned_c4(args, local_rank):
    """The learned initial guess at the stated learned-guess workload: the
    graph network is trained on `--c4-train` solved ensembles (N ~ U[1000,
    5000], lmax 3, fill ~ U[0.2, 0.4], R = 100 nm, n = 1.52, x-polarised plane
    wave), then 100 unseen ensembles of 8000 spheres are solved from T a and
    from the learned first iterate (mixed precision to 1e-6): GMRES
    iterations, time (prediction included) and the final FP64 residual.
    Packings are made by spawn workers on the host cores while the GPU solves.
    Evaluation seeds (index 100 000 + e) are disjoint from training seeds."""
    import multiprocessing as mp
    import synth
    from paper_1706_02145_gb300 import binding as B
    cores = host_cores()
    n_train, n_eval, epochs = args.c4_train, args.c4_eval, args.c4_epochs
    out = {"train_ensembles": n_train, "eval_ensembles": n_eval, "epochs": epochs, "width": 128, "layers": 3,
           "knn": 16, "eval_N": 8000}
    g = B.celes_gnn_create(3, width=128, layers=3, seed=1, device=local_rank)
    try:
        t0 = time.perf_counter()
        t_gpu = 0.0
        train_its = []
        with mp.get_context("spawn").Pool(max(1, cores - 1)) as pool:
            for idx, pos, rad, nn, name in pool.imap_unordered(_pack_config4, range(n_train), chunksize=4):
                tg = time.perf_counter()
                c = B.celes_create(pos, rad, nn, 1.0, 2 * np.pi / 550.0, 3, device=local_rank)
                try:
                    B.celes_set_incident(c, [B.make_incident("plane", beta=0.0, alpha=0.0, pol=2)])
                    info = B.celes_solve(c, 1e-7, mode=B.CELES_SOLVE_MIXED, raise_on_noconv=False)
                    train_its.append(info["iterations"])
                    B.celes_gnn_add_example(g, c)
                finally:
                    B.celes_destroy(c)
                t_gpu += time.perf_counter() - tg
            out["data_s"] = time.perf_counter() - t0
            out["data_gpu_s"] = t_gpu
            out["train_mean_iterations"] = float(np.mean(train_its))
            # training: epochs over the stored examples in a seeded random order
            rng = np.random.default_rng(3)
            t0 = time.perf_counter()
            losses = []
            for ep in range(epochs):
                lr = 1e-3 * (0.5 ** (ep // max(1, epochs // 4)))
                ls = [B.celes_gnn_train_example(g, int(i), steps=1, lr=lr) for i in rng.permutation(n_train)]
                losses.append(float(np.mean(ls)))
            out["train_s"] = time.perf_counter() - t0
            out["loss_per_epoch"] = losses
            B.celes_gnn_clear_examples(g)
            # evaluation on unseen 8000-sphere ensembles
            rows = []
            t0 = time.perf_counter()
            for idx, pos, rad, nn, name in pool.imap(partial(_pack_config4, N=8000),
                                                     [100_000 + e for e in range(n_eval)]):
                c = B.celes_create(pos, rad, nn, 1.0, 2 * np.pi / 550.0, 3, device=local_rank)
                try:
                    B.celes_set_incident(c, [B.make_incident("plane", beta=0.0, alpha=0.0, pol=2)])
                    base = B.celes_solve(c, TOL, mode=B.CELES_SOLVE_MIXED, raise_on_noconv=False)
                    tp = time.perf_counter()
                    B.celes_gnn_predict(g, c)
                    t_pred = time.perf_counter() - tp
                    lg = B.celes_solve(c, TOL, mode=B.CELES_SOLVE_MIXED, x0=B.CELES_X0_LEARNED,
                                       raise_on_noconv=False)
                    rows.append((base["iterations"], lg["iterations"], base["seconds"], lg["seconds"] + t_pred,
                                 base["residual"], lg["residual"], lg["guess_used"], name))
                finally:
                    B.celes_destroy(c)
            out["eval_s"] = time.perf_counter() - t0
        its_b = np.array([r[0] for r in rows], float)
        its_l = np.array([r[1] for r in rows], float)
        out.update({"ta_mean_iterations": float(its_b.mean()), "learned_mean_iterations": float(its_l.mean()),
                    "mean_iterations_saved": float((its_b - its_l).mean()),
                    "ta_mean_s": float(np.mean([r[2] for r in rows])),
                    "learned_mean_s": float(np.mean([r[3] for r in rows])),
                    "max_final_residual": float(max(max(r[4], r[5]) for r in rows)),
                    "guess_used_fraction": float(np.mean([r[6] for r in rows])),
                    "per_ensemble": [{"ta_its": r[0], "learned_its": r[1], "name": r[7]} for r in rows[:20]]})
        return out
    finally:
        B.celes_gnn_destroy(g)


def run_c5(args, local_rank):
    """The large workload end to end: 100 000 monodisperse spheres (R = 130
    nm, n = 1.52, lmax 3) in a 4 um slab at fill 0.25, Gaussian beam of waist
    5 um, the paper's block-diagonal preconditioner over 1 um cuboids
    (Sec. 3.2.1), FP32 inner GMRES with FP64 refinement to 1e-6.  Reports the
    packing, incident, preconditioner build and solve times, iterations, the
    FP32 coupling matvec and preconditioner-apply times (CUDA events; the
    apply as a fraction of the measured HBM bandwidth) and the oracle's
    residual of the solution on sampled receiver rows (cpu_baseline leg)."""
    import torch
    import synth
    from paper_1706_02145_gb300 import binding as B
    out = {"workload": "100 000 spheres R=130nm n=1.52 lmax 3, 4um slab fill 0.25, Gaussian w=5um, "
                       f"block-diagonal preconditioner {args.c5_edge:g} nm cuboids, mixed solve to 1e-6"}
    t0 = time.perf_counter()
    sc = synth.config5(0)
    out["pack_s"] = time.perf_counter() - t0
    inc_d = sc.incidents[0]
    inc = B.make_incident("gaussian", waist=inc_d.waist, focus=inc_d.focus, alpha_G=inc_d.alpha_G, n_beta=128)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax, device=local_rank)
    try:
        t0 = time.perf_counter()
        B.celes_set_incident(ctx, [inc])
        torch.cuda.synchronize()
        out["incident_s"] = time.perf_counter() - t0

        # a stream of its own: the binding passes NULL for the legacy default
        # stream, which would launch on the context's stream instead
        st = torch.cuda.Stream()

        def timed(fn, reps):
            fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(reps):
                fn()
            b.record(st)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        g = torch.Generator(device="cuda").manual_seed(0)
        x = torch.randn(sc.N, sc.nmax, dtype=torch.complex64, device="cuda", generator=g)
        y = torch.empty_like(x)
        ms_mv = timed(lambda: B.celes_coupling_matvec(ctx, x, y, precision=B.CELES_FP32, stream=st), 3)
        out["matvec_fp32_ms"] = ms_mv
        out["matvec_fp32_couplings_per_s"] = sc.N * (sc.N - 1) / (ms_mv / 1e3)
        t0 = time.perf_counter()
        B.celes_precond_build(ctx, args.c5_edge)
        out["precond_build_s"] = time.perf_counter() - t0
        nb, maxd, ent = B.celes_precond_stats(ctx)
        ms_ap = timed(lambda: B.celes_precond_apply(ctx, x, y, precision=B.CELES_FP32, stream=st), 5)
        gbs = ent * 8 / (ms_ap / 1e3) / 1e9
        hbm = None
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                hbm = json.load(fh).get("hbm_gbs")
        except Exception:
            pass
        out["precond"] = {"blocks": nb, "max_block_dim": maxd, "factor_bytes_fp32": ent * 8,
                          "factor_bytes_fp64": ent * 16, "apply_fp32_ms": ms_ap, "apply_gbs": gbs,
                          "apply_frac_of_measured_hbm": (gbs / hbm) if hbm else None}
        info = B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_MIXED, use_precond=True, max_iter=20000,
                             raise_on_noconv=False)
        out["solve"] = {"s": info["seconds"], "iterations": info["iterations"], "outer": info["outer"],
                        "matvecs_fp32": info["matvecs_fp32"], "matvecs_fp64": info["matvecs_fp64"],
                        "residual_fp64_gpu": info["residual"], "status": info["status"]}
        out["total_s"] = out["incident_s"] + out["precond_build_s"] + info["seconds"]
        b = B.celes_get_coefficients(ctx)[0]
    finally:
        B.celes_destroy(ctx)
    if not args.no_cpu:
        import multiprocessing as mp
        cores = host_cores()
        rows = [int(r) for r in np.random.default_rng(11).choice(sc.N, 4 * cores, replace=False)]
        with mp.get_context("spawn").Pool(cores) as pool:
            (res,), rate, dt = certify_rows(sc, inc_d, [b], rows, cores, pool)
        out["oracle_sampled_residual"] = {"rows": len(rows), "residual": res, "oracle_couplings_per_s": rate,
                                          "oracle_s": dt, "cores": cores}
    return out


def run_plain_full(args, local_rank):
    """The plain FP64 GMRES solve of the full bench workload to 1e-6,
    uncapped (about 10 min), beside the chosen form (FP32 inner GMRES with
    FP64 refinement) on the same context; both errors against the same
    system refined to 1e-10."""
    import synth
    from paper_1706_02145_gb300 import binding as B
    scene = synth.config2(0, N=args.N)
    d = scene.incidents[0]
    inc = B.make_incident("gaussian", waist=d.waist, focus=d.focus, alpha_G=d.alpha_G, n_beta=128)
    ctx = B.celes_create(scene.positions, scene.radii, scene.n_sphere, scene.n0, scene.k0, scene.lmax,
                         device=local_rank)
    try:
        B.celes_set_incident(ctx, [inc])
        B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_MIXED)  # warm-up (and the tuner)
        ic = B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_MIXED)
        bc = B.celes_get_coefficients(ctx)[0]
        ir = B.celes_solve(ctx, REF_TOL, mode=B.CELES_SOLVE_MIXED, max_iter=40000, max_outer=40,
                           raise_on_noconv=False)
        br = B.celes_get_coefficients(ctx)[0]
        ip = B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_FP64, max_iter=20000, use_precond=False,
                           raise_on_noconv=False)
        bp = B.celes_get_coefficients(ctx)[0]
    finally:
        B.celes_destroy(ctx)
    return {"N": scene.N, "lmax": scene.lmax,
            "chosen": {"s": ic["seconds"], "iterations": ic["iterations"], "residual": ic["residual"],
                       "error_vs_reference": rel_err(bc, br)},
            "plain_fp64": {"s": ip["seconds"], "iterations": ip["iterations"], "residual": ip["residual"],
                           "status": ip["status"], "error_vs_reference": rel_err(bp, br)},
            "reference": {"tol": REF_TOL, "residual": ir["residual"], "iterations": ir["iterations"]},
            "speedup": ip["seconds"] / ic["seconds"]}


def max_over_ranks(x, dist, device):
    """The largest of a per-rank scalar (every rank gets it)."""
    if not dist:
        return float(x)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, max_ms):
    """Whole-job throughput of replicas: the units all ranks processed over
    the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def measure_peaks():
    """FP32 and FP64 FMA issue peaks of this GPU, measured by the library's
    FMA-chain kernels (celes_fma_peak) right before the timed steps."""
    from paper_1706_02145_gb300 import binding as B
    f32, _ = B.celes_fma_peak(B.FMA_FP32)
    f32p, _ = B.celes_fma_peak(B.FMA_FP32_PACKED)
    f64, _ = B.celes_fma_peak(B.FMA_FP64)
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    return {"fp32_tflops": max(f32, f32p), "fp32_scalar_tflops": f32, "fp32_packed_tflops": f32p,
            "fp64_tflops": f64, "sms": props.multi_processor_count,
            "how": "celes_fma_peak: 16 independent FMA chains per thread, 4 x 256 threads per SM, best of 3 "
                   "CUDA-event-timed launches, at the SM clock of that moment"}


def certify_rows(scene, inc, vectors, rows, cores, pool=None):
    """The oracle's FP64 residual of candidate solutions on sampled receiver
    rows (part of the cpu_baseline leg, whose timed work is the same
    on-the-fly coupling rows): r_S = (T a)_S - b_S + T_S (W b)_S, relative to
    ||(T a)_S||, with T (App. B) and a (App. C, the same 128-node beta rule)
    from the oracle.  Returns (relative residual per vector, oracle
    couplings/s, seconds of coupling-row work)."""
    from oracle import incident, mie
    rows = list(rows)
    t = mie.t_diagonal(scene.lmax, scene.k, scene.radii[rows], scene.n_rel[rows])
    a = incident.gaussian_beam_coeffs(scene.lmax, scene.k, scene.positions[rows], inc.waist, inc.focus,
                                      inc.alpha_G, n_beta=128)
    ta = t * a
    res, t_total, pairs = [], 0.0, 0
    for b in vectors:
        wb, dt = oracle_rows(scene, b, rows, cores, pool)
        t_total += dt
        pairs += len(rows) * (scene.N - 1)
        r = ta - b[rows] + t * wb
        res.append(float(np.linalg.norm(r) / np.linalg.norm(ta)))
    return res, pairs / t_total, t_total


def oracle_rows(scene, x, rows, n_workers, pool=None):
    """(W x)_rows by the oracle's on-the-fly FP64 coupling rows in spawn
    workers: (values (len(rows), nmax), seconds)."""
    import multiprocessing as mp
    chunks = [list(rows[q::n_workers]) for q in range(n_workers)]
    idx = [q for q in range(n_workers) if chunks[q]]
    args = [(scene.positions, scene.k, scene.lmax, x, chunks[q]) for q in idx]
    t0 = time.perf_counter()
    if pool is None:
        with mp.get_context("spawn").Pool(len(args)) as p:
            parts = p.starmap(_oracle_rows_values, args)
    else:
        parts = pool.starmap(_oracle_rows_values, args)
    dt = time.perf_counter() - t0
    out = np.zeros((len(rows), scene.nmax), dtype=complex)
    pos_of = {r: q for q, r in enumerate(rows)}
    for q, part in zip(idx, parts):
        for r, v in zip(chunks[q], part):
            out[pos_of[r]] = v
    return out, dt


def _oracle_rows_values(pos, k, lmax, x, rows):
    from oracle import translation
    return translation.coupling_matvec_rows(pos, k, lmax, x, rows)


def rel_err(b, ref):
    return float(np.linalg.norm(b - ref) / np.linalg.norm(ref))


def run_ours(args, rank, world, local_rank):
    import torch
    import synth
    from paper_1706_02145_gb300 import binding as B

    torch.cuda.set_device(local_rank)
    if not os.path.exists(B.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    B.load()
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    scene = synth.config2(0, N=args.N)
    N, L = scene.N, scene.lmax
    pairs = N * (N - 1)
    inc_desc = scene.incidents[0]
    inc = B.make_incident("gaussian", waist=inc_desc.waist, focus=inc_desc.focus, alpha_G=inc_desc.alpha_G,
                          n_beta=128)
    bb, aa = np.meshgrid(np.linspace(0.0, np.pi, 32), np.linspace(0.0, 2 * np.pi, 64, endpoint=False),
                         indexing="ij")
    dirs = np.stack([bb.ravel(), aa.ravel()], axis=1)

    ctx = B.celes_create(scene.positions, scene.radii, scene.n_sphere, scene.n0, scene.k0, L, device=local_rank)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        B.celes_set_incident(ctx, [inc])
        info = B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_MIXED)
        B.celes_farfield(ctx, dirs)
        return info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    peaks = measure_peaks()

    B.celes_profile(ctx, 1)
    sampler = ClockSampler(local_rank)
    sampler.start()
    launches0 = B.celes_kernel_launches()
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    for q in range(args.steps):
        flush.fill_(float(q))
        ev[q][0].record(st)
        infos.append(step())
        ev[q][1].record(st)
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    launches = B.celes_kernel_launches() - launches0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    mv32 = sum(i["matvecs_fp32"] for i in infos)
    mv64 = sum(i["matvecs_fp64"] for i in infos)
    value = job_value((mv32 + mv64) * pairs, world, total_ms)
    b_chosen = B.celes_get_coefficients(ctx)[0]

    # kernel-level roofline from the library's CUDA events (on the launch stream)
    fpp = flops_per_pair(L)
    k32_ms, k32_n = B.celes_kernel_time(ctx, B.KERNEL_FP32_COUPLING)
    k64_ms, k64_n = B.celes_kernel_time(ctx, B.KERNEL_FP64_COUPLING)
    ep_ms, ep_n = B.celes_kernel_time(ctx, B.KERNEL_EPILOGUE)
    B.celes_profile(ctx, 0)
    kernels = {
        "coupling_fp32": {"ms": k32_ms, "launches": k32_n,
                          "tflops": (fpp * pairs * k32_n / (k32_ms / 1e3) / 1e12) if k32_n else None,
                          "couplings_per_s": (pairs * k32_n / (k32_ms / 1e3)) if k32_n else None},
        "coupling_fp64": {"ms": k64_ms, "launches": k64_n,
                          "tflops": (fpp * pairs * k64_n / (k64_ms / 1e3) / 1e12) if k64_n else None,
                          "couplings_per_s": (pairs * k64_n / (k64_ms / 1e3)) if k64_n else None},
        "epilogue": {"ms": ep_ms, "launches": ep_n},
    }
    for key, pk in (("coupling_fp32", peaks["fp32_tflops"]), ("coupling_fp64", peaks["fp64_tflops"])):
        tf = kernels[key]["tflops"]
        kernels[key]["frac_of_measured_peak"] = (tf / pk) if tf else None
    for key, prec in (("coupling_fp32", B.CELES_FP32), ("coupling_fp64", B.CELES_FP64)):
        try:
            v, ch, tms = B.celes_coupling_shape(ctx, prec)
            kernels[key]["shape"] = {"variant": v, "chunks": ch, "tuned_ms": tms}
        except B.CelesError:
            pass
    dom = "coupling_fp32" if k32_ms >= k64_ms else "coupling_fp64"
    peak = peaks["fp32_tflops"] if dom == "coupling_fp32" else peaks["fp64_tflops"]
    ach = kernels[dom]["tflops"]
    shp = kernels[dom].get("shape")
    traffic = ncu_traffic(f"{dom}_L{L}", (shp["variant"], shp["chunks"]) if shp else None)
    derived = peaks["sms"] * 128 * 2 * 2.070e9 / 1e12
    roofline = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": (ach / peak) if ach else None, "traffic": traffic, "kernel": dom,
                "flops_per_pair": fpp,
                "peak_basis": (f"measured {'FP32' if dom == 'coupling_fp32' else 'FP64'} FMA issue peak of this GPU "
                               "(celes_fma_peak, run just before the timed steps)"),
                "measured_peaks": peaks,
                "fp32_derived_peak_tflops": derived,
                "frac_of_derived_fp32_peak": (kernels["coupling_fp32"]["tflops"] / derived)
                if kernels["coupling_fp32"]["tflops"] else None,
                "direct_method_flops_per_pair": B.celes_flops_per_pair(L, B.CELES_KERNEL_DIRECT),
                "share_of_step": (kernels[dom]["ms"] / total_ms) if total_ms else None}

    # chosen form vs plain FP64: time to 1e-6 on the same inputs
    tt = {"chosen_s": float(np.mean([i["seconds"] for i in infos])),
          "chosen_iterations": infos[-1]["iterations"], "chosen_matvecs_fp32": infos[-1]["matvecs_fp32"],
          "chosen_matvecs_fp64": infos[-1]["matvecs_fp64"], "chosen_residual": infos[-1]["residual"]}
    b_ref = None
    if not args.no_certify:
        # the reference: the same system refined in FP64 to 1e-10 (certified
        # below by the oracle's residual on sampled rows)
        ir = B.celes_solve(ctx, REF_TOL, mode=B.CELES_SOLVE_MIXED, max_iter=40000, max_outer=40,
                           raise_on_noconv=False)
        b_ref = B.celes_get_coefficients(ctx)[0]
        tt["reference"] = {"tol": REF_TOL, "residual_fp64_gpu": ir["residual"], "iterations": ir["iterations"],
                           "matvecs_fp64": ir["matvecs_fp64"], "s": ir["seconds"],
                           "how": "FP32 GMRES inner solves with FP64 residuals (iterative refinement) to 1e-10"}
        tt["error_vs_fp64_oracle"] = rel_err(b_chosen, b_ref)
    others = {}
    if not args.no_precond:
        # the paper's block-diagonal preconditioner (Sec. 3.2.1) on the same
        # solve: fewer coupling matvecs for a build and an apply per iteration
        pre = {}
        for edge in (600.0, 900.0):
            t0 = time.perf_counter()
            B.celes_precond_build(ctx, edge)
            tb = time.perf_counter() - t0
            ip = B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_MIXED, use_precond=True)
            e = {"build_s": tb, "solve_s": ip["seconds"], "total_s": tb + ip["seconds"],
                 "iterations": ip["iterations"], "residual": ip["residual"]}
            if b_ref is not None:
                e["error_vs_fp64_oracle"] = rel_err(B.celes_get_coefficients(ctx)[0], b_ref)
            pre[f"edge_{int(edge)}nm"] = e
        tt["block_preconditioned"] = pre
    if not args.no_plain:
        # (b) measured end to end on a reduced packing of the same recipe
        small = synth.config2(0, N=args.small_n)
        cs = B.celes_create(small.positions, small.radii, small.n_sphere, small.n0, small.k0, L, device=local_rank)
        try:
            B.celes_set_incident(cs, [inc])
            B.celes_solve(cs, TOL, mode=B.CELES_SOLVE_MIXED)  # warm-up
            im = B.celes_solve(cs, TOL, mode=B.CELES_SOLVE_MIXED)
            bm = B.celes_get_coefficients(cs)[0]
            ip = B.celes_solve(cs, TOL, mode=B.CELES_SOLVE_FP64, raise_on_noconv=False)
            bp = B.celes_get_coefficients(cs)[0]
            ib = B.celes_solve(cs, TOL, mode=B.CELES_SOLVE_MIXED, solver=B.CELES_SOLVER_BICGSTAB,
                               raise_on_noconv=False)
            bb = B.celes_get_coefficients(cs)[0]
            ms = {"N": small.N, "chosen_s": im["seconds"], "chosen_iterations": im["iterations"],
                  "plain_fp64_s": ip["seconds"], "plain_fp64_iterations": ip["iterations"],
                  "plain_fp64_residual": ip["residual"], "chosen_residual": im["residual"],
                  "speedup": ip["seconds"] / im["seconds"],
                  "chosen_vs_plain_rel_l2": rel_err(bm, bp),
                  "bicgstab_mixed": {"s": ib["seconds"], "iterations": ib["iterations"],
                                     "matvecs_fp32": ib["matvecs_fp32"], "residual": ib["residual"],
                                     "vs_plain_rel_l2": rel_err(bb, bp)}}
            if not args.no_certify:
                ir = B.celes_solve(cs, REF_TOL, mode=B.CELES_SOLVE_MIXED, max_iter=40000, max_outer=40,
                                   raise_on_noconv=False)
                bs_ref = B.celes_get_coefficients(cs)[0]
                ms["reference_residual_fp64_gpu"] = ir["residual"]
                ms["error_vs_fp64_oracle"] = rel_err(bm, bs_ref)
                ms["plain_fp64_error_vs_fp64_oracle"] = rel_err(bp, bs_ref)
                ms["bicgstab_mixed"]["error_vs_fp64_oracle"] = rel_err(bb, bs_ref)
                others["small"] = (small, bm, bs_ref)
            tt["measured_small"] = ms
        finally:
            B.celes_destroy(cs)
        # (a) full size: plain FP64 GMRES for a bounded number of iterations
        #     gives its time per iteration; its time to 1e-6 is extrapolated
        #     with (i) the chosen form's iteration count and (ii) that count
        #     scaled by plain/chosen iterations measured at the small size
        cap = 24
        info_p = B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_FP64, max_iter=cap, use_precond=False,
                                raise_on_noconv=False)
        per_it = info_p["seconds"] / max(1, info_p["iterations"])
        ratio = ms["plain_fp64_iterations"] / max(1, ms["chosen_iterations"])
        tt["plain_fp64_s_per_iteration"] = per_it
        tt["plain_fp64_s_extrapolated"] = per_it * tt["chosen_iterations"]
        tt["plain_fp64_s_extrapolated_scaled"] = per_it * tt["chosen_iterations"] * ratio
        tt["speedup_extrapolated"] = tt["plain_fp64_s_extrapolated"] / tt["chosen_s"]
        tt["speedup_extrapolated_scaled"] = tt["plain_fp64_s_extrapolated_scaled"] / tt["chosen_s"]
        tt["extrapolation"] = (f"plain FP64 GMRES timed for {info_p['iterations']} iterations at full size, times "
                               f"(i) the {tt['chosen_iterations']} iterations of the chosen form, (ii) that count "
                               f"times the plain/chosen iteration ratio {ratio:.3f} measured at N={small.N}")
        if args.plain_full:
            ipf = B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_FP64, max_iter=20000, use_precond=False,
                                raise_on_noconv=False)
            tt["plain_fp64_full"] = {"s": ipf["seconds"], "iterations": ipf["iterations"],
                                     "residual": ipf["residual"], "speedup": ipf["seconds"] / tt["chosen_s"]}
            if b_ref is not None:
                tt["plain_fp64_full"]["error_vs_fp64_oracle"] = rel_err(B.celes_get_coefficients(ctx)[0], b_ref)
    B.celes_destroy(ctx)
    batched = None if args.no_batched else run_batched(args, local_rank)
    learned = None if args.no_learned else run_learned(args, local_rank)

    # end to end through the C ABI with host buffers: H2D of the inputs,
    # D2H of the coefficients, every step
    e2e = None
    if not args.no_e2e:
        h2d = scene.positions.nbytes + scene.radii.nbytes + scene.n_sphere.astype(np.complex128).nbytes
        d2h = N * scene.nmax * 16
        e2e_ms = []
        e2e_mv = 0
        for q in range(args.steps):
            flush.fill_(float(q))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c2 = B.celes_create(scene.positions, scene.radii, scene.n_sphere, scene.n0, scene.k0, L,
                                device=local_rank)
            B.celes_set_incident(c2, [inc])
            inf = B.celes_solve(c2, TOL, mode=B.CELES_SOLVE_MIXED)
            B.celes_get_coefficients(c2)
            B.celes_farfield(c2, dirs)
            B.celes_destroy(c2)
            torch.cuda.synchronize()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
            e2e_mv += inf["matvecs_fp32"] + inf["matvecs_fp64"]
        e2e_total = max_over_ranks(float(sum(e2e_ms)), dist, "cuda")
        e2e = {"value": job_value(e2e_mv * pairs, world, e2e_total), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h + dirs.shape[0] * 32), "ms_per_step": e2e_total / args.steps}

    cpu = None
    if rank == 0 and not args.no_cpu and world == 1:
        # the oracle timed on the host cores: its on-the-fly FP64 coupling rows
        # on a sample of receivers of the workload.  When the certified
        # reference exists, the sampled rows are applied to the chosen and the
        # reference solutions, and the same rows give the oracle's residual of
        # both (the certification of the reference).
        import multiprocessing as mp
        cores = host_cores()
        rows = args.cpu_rows or 16 * max(cores, 2)
        sel = [int(r) for r in np.random.default_rng(7).choice(N, rows, replace=False)]
        with mp.get_context("spawn").Pool(cores) as pool:
            if b_ref is not None:
                (r_chosen, r_ref), rate, dt = certify_rows(scene, inc_desc, [b_chosen, b_ref], sel, cores, pool)
                tt["oracle_sampled_residual"] = {"rows": rows, "chosen": r_chosen, "reference": r_ref}
                if "small" in others:
                    small, bm, bs_ref = others["small"]
                    ssel = [int(r) for r in np.random.default_rng(8).choice(small.N, 4 * cores, replace=False)]
                    (rs_c, rs_r), _, _ = certify_rows(small, inc_desc, [bm, bs_ref], ssel, cores, pool)
                    tt["measured_small"]["oracle_sampled_residual"] = {"rows": len(ssel), "chosen": rs_c,
                                                                       "reference": rs_r}
                what = "the chosen and the reference solution"
            else:
                x = np.random.default_rng(1).normal(size=(N, scene.nmax)) * (1 + 0j)
                _, dt = oracle_rows(scene, x, sel, cores, pool)
                rate = rows * (N - 1) / dt
                what = "a random vector"
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{rows} receiver rows x {N - 1} sources of the oracle's FP64 on-the-fly coupling "
                         f"matvec applied to {what} (numpy, {cores} spawn workers), {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": workload_config(N, L, world),
                "roofline": roofline, "kernels": kernels, "time_to_1e-6": tt, "batched": batched,
                "learned_guess": learned, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks}
        print(json.dumps(line), flush=True)


def run_case(args):
    """One hot-path operation on a synthetic case, through the C ABI, for
    timing and profiling (ncu captures of single launches):
      coupling: y = W x on the bench recipe with --N spheres and --lmax (or the
                100 000-sphere slab, --recipe large); --rhs right-hand sides;
      precond:  builds the block-diagonal preconditioner with --edge nm cuboids
                on the same recipe and applies it;
      batch:    the batched operator (I - T W) over --ensembles ensembles of
                the multi-ensemble recipe (sizes scaled by 0.4), --rhs plane
                waves each.
    Runs --reps operations and prints the time of the last one."""
    import torch
    import synth
    from paper_1706_02145_gb300 import binding as B
    B.load()
    prec = B.CELES_FP32 if args.precision == "fp32" else B.CELES_FP64
    dt = torch.complex64 if prec == B.CELES_FP32 else torch.complex128
    g = torch.Generator(device="cuda").manual_seed(0)
    if args.case == "batch":
        nrhs = args.rhs or 4
        scenes = [synth.config3(e, n_rhs=nrhs, N=max(80, int(0.4 * synth.config3_size(e))))
                  for e in range(args.ensembles)]
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
        for _ in range(args.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B.celes_batch_master_matvec(bt, x, y, precision=prec)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
        pairs = sum(sc.N * (sc.N - 1) * len(sc.incidents) for sc in scenes)
        print(f"batch of {len(scenes)} ensembles x {nrhs} RHS, {args.precision}: {t * 1e3:.3f} ms, "
              f"{pairs / t:.3e} couplings/s")
        B.celes_batch_destroy(bt)
        for c in ctxs:
            B.celes_destroy(c)
        return
    if args.case == "solve":
        # the mixed solve of the bench workload (--N spheres, --lmax) to 1e-6
        # for each inner tolerance: time, iterations and FP64 matvecs
        sc = synth.config2(0, N=args.N, lmax=args.lmax)
        d = sc.incidents[0]
        ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax)
        B.celes_set_incident(ctx, [B.make_incident("gaussian", waist=d.waist, focus=d.focus, alpha_G=d.alpha_G,
                                                   n_beta=128)])
        B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_MIXED)  # warm-up (and the tuner)
        for it in [float(v) for v in args.inner_tol.split(",")]:
            info = B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_MIXED, inner_tol=it, raise_on_noconv=False)
            print(f"N={sc.N} lmax={sc.lmax} mixed solve to {TOL:g}, inner tol {it:g}: {info['seconds']:.3f} s, "
                  f"{info['iterations']} iterations, {info['matvecs_fp32']} FP32 and {info['matvecs_fp64']} FP64 "
                  f"matvecs, residual {info['residual']:.3e}, status {info['status']}")
        B.celes_destroy(ctx)
        return
    kern = {"auto": B.CELES_KERNEL_AUTO, "direct": B.CELES_KERNEL_DIRECT, "rtr": B.CELES_KERNEL_RTR}[args.kernel]
    sc = synth.config2(0, N=args.N, lmax=args.lmax) if args.recipe == "slab" else synth.config5(0)
    ctx = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax, kernel=kern,
                         autotune=bool(args.autotune), variant=args.variant, chunks=args.chunks)
    nrhs = max(1, args.rhs) if args.case == "coupling" else 1
    x = torch.randn(nrhs, sc.N, sc.nmax, dtype=dt, device="cuda", generator=g)
    y = torch.empty_like(x)
    if args.case == "precond":
        B.celes_precond_build(ctx, args.edge)
    t = 0.0
    for _ in range(args.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if args.case == "precond":
            B.celes_precond_apply(ctx, x, y, precision=prec)
        else:
            B.celes_coupling_matvec(ctx, x, y, nrhs=nrhs, precision=prec)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    if args.case == "precond":
        nb, maxd, ent = B.celes_precond_stats(ctx)
        fb = ent * (8 if prec == B.CELES_FP32 else 16)
        print(f"N={sc.N} lmax={sc.lmax} {args.precision} block preconditioner apply (edge {args.edge:g} nm, "
              f"{nb} blocks, largest {maxd}): {t * 1e3:.3f} ms, factors {fb / 1e9:.3f} GB, {fb / t / 1e9:.1f} GB/s")
    else:
        pairs = sc.N * (sc.N - 1) * nrhs
        shape = B.celes_coupling_shape(ctx, prec) if args.kernel != "direct" else None
        kern_id = B.CELES_KERNEL_DIRECT if args.kernel == "direct" else B.CELES_KERNEL_RTR
        tflops = B.celes_flops_per_pair(sc.lmax, kern_id) * pairs / t / 1e12
        peak, _ = B.celes_fma_peak(B.FMA_FP32 if prec == B.CELES_FP32 else B.FMA_FP64)
        print(f"N={sc.N} lmax={sc.lmax} {args.precision} kernel={args.kernel} rhs={nrhs}: {t * 1e3:.3f} ms, "
              f"{pairs / t:.3e} couplings/s, {tflops:.1f} TFLOP/s = {tflops / peak:.3f} of the measured "
              f"{peak:.1f}, shape (variant, chunks, tuned ms) {shape}")
    B.celes_destroy(ctx)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.case:
        run_case(args)
        return
    if args.plain_full_only:
        import torch
        torch.cuda.set_device(local_rank)
        from paper_1706_02145_gb300 import binding as B
        B.load()
        print(json.dumps({"plain_fp64_full": run_plain_full(args, local_rank)}), flush=True)
        return
    if args.c5:
        import torch
        torch.cuda.set_device(local_rank)
        from paper_1706_02145_gb300 import binding as B
        B.load()
        print(json.dumps({"large_c5": run_c5(args, local_rank)}), flush=True)
        return
    if args.learned_c4:
        import torch
        torch.cuda.set_device(local_rank)
        from paper_1706_02145_gb300 import binding as B
        B.load()
        print(json.dumps({"learned_guess_c4": run_learned_c4(args, local_rank)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
