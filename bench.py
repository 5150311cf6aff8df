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

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sphere-pair couplings/s; time to 1e-6 residual, chosen form vs plain FP64"
UNIT = "sphere-pair couplings/s"
TOL = 1e-6
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12      # SMs x FP32 lanes x FMA x max SM clock
FP64_PEAK_TFLOPS = 1.25                                   # nominal GB300 FP64


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
    ap.add_argument("--batched-ensembles", type=int, default=12)
    ap.add_argument("--batched-rhs", type=int, default=4)
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-initial-guess measurement")
    ap.add_argument("--no-precond", action="store_true", help="skip the block-preconditioned solve")
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


def ncu_traffic(kernel_key):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or
    None when it is absent or was taken on other kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(kernel_key)
        if e and e.get("source_hash") == kernel_source_hash():
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

def run_batched(args, local_rank):
    """Many uneven ensembles x RHS in one lockstep batched solve against the
    same systems solved one context at a time (ensembles of the multi-ensemble
    recipe: lmax 2..5, plane waves from a 60 degree cap; sizes scaled by 0.4
    so the measurement takes seconds)."""
    import torch
    import synth
    from paper_1706_02145_gb300 import binding as B
    scenes = []
    for e in range(args.batched_ensembles):
        scenes.append(synth.config3(e, n_rhs=args.batched_rhs, N=max(80, int(0.4 * synth.config3_size(e)))))
    ctxs = []
    try:
        for sc in scenes:
            c = B.celes_create(sc.positions, sc.radii, sc.n_sphere, sc.n0, sc.k0, sc.lmax, device=local_rank)
            ctxs.append(c)
            B.celes_set_incident(c, [B.make_incident("plane", beta=i.beta, alpha=i.alpha, pol=i.pol)
                                     for i in sc.incidents])
        bt = B.celes_batch_create(ctxs, restart=30)
        try:
            n = B.celes_batch_num_unknowns(bt)
            x = torch.ones(n, dtype=torch.complex64, device=f"cuda:{local_rank}")
            y = torch.empty_like(x)
            B.celes_batch_master_matvec(bt, x, y, precision=B.CELES_FP32)  # graph capture, warm-up
            reps = 5
            t0 = time.perf_counter()
            for _ in range(reps):
                B.celes_batch_master_matvec(bt, x, y, precision=B.CELES_FP32)
            t_mv = (time.perf_counter() - t0) / reps
            pairs = sum(sc.N * (sc.N - 1) * len(sc.incidents) for sc in scenes)
            code, infos = B.celes_batch_solve(bt, len(ctxs), TOL, mode=B.CELES_SOLVE_MIXED, restart=30,
                                              raise_on_noconv=False)
            t_batch = max(i["seconds"] for i in infos)
            res_batch = max(i["residual"] for i in infos)
            its_batch = max(i["iterations"] for i in infos)
        finally:
            B.celes_batch_destroy(bt)
        t_one, res_one = 0.0, 0.0
        for c in ctxs:
            info = B.celes_solve(c, TOL, mode=B.CELES_SOLVE_MIXED, restart=30, use_precond=False,
                                 raise_on_noconv=False)
            t_one += info["seconds"]
            res_one = max(res_one, info["residual"])
        return {"ensembles": len(scenes), "rhs_each": args.batched_rhs, "systems": len(scenes) * args.batched_rhs,
                "N_range": [min(sc.N for sc in scenes), max(sc.N for sc in scenes)],
                "lmax_values": sorted({sc.lmax for sc in scenes}),
                "operator_fp32_ms": t_mv * 1e3, "operator_couplings_per_s": pairs / t_mv,
                "batched_solve_s": t_batch, "batched_max_iterations": its_batch, "batched_max_residual": res_batch,
                "one_by_one_solve_s": t_one, "one_by_one_max_residual": res_one, "speedup": t_one / t_batch,
                "note": "mixed FP32/FP64 GMRES(30) to 1e-6, no preconditioner, first iterate T a, both forms"}
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
    dom = "coupling_fp32" if k32_ms >= k64_ms else "coupling_fp64"
    peak = FP32_PEAK_TFLOPS if dom == "coupling_fp32" else FP64_PEAK_TFLOPS
    ach = kernels[dom]["tflops"]
    traffic = ncu_traffic(f"{dom}_L{L}")
    roofline = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": (ach / peak) if ach else None, "traffic": traffic, "kernel": dom,
                "flops_per_pair": fpp,
                "peak_basis": ("152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz max SM clock" if dom == "coupling_fp32"
                               else "nominal GB300 FP64 1.25 TFLOP/s"),
                "direct_method_flops_per_pair": B.celes_flops_per_pair(L, B.CELES_KERNEL_DIRECT),
                "share_of_step": (kernels[dom]["ms"] / total_ms) if total_ms else None}

    # chosen form vs plain FP64: time to 1e-6 on the same inputs
    tt = {"chosen_s": float(np.mean([i["seconds"] for i in infos])),
          "chosen_iterations": infos[-1]["iterations"], "chosen_matvecs_fp32": infos[-1]["matvecs_fp32"],
          "chosen_matvecs_fp64": infos[-1]["matvecs_fp64"], "chosen_residual": infos[-1]["residual"]}
    if not args.no_precond:
        # the paper's block-diagonal preconditioner (Sec. 3.2.1) on the same
        # solve: fewer coupling matvecs for a build and an apply per iteration
        pre = {}
        for edge in (600.0, 900.0):
            t0 = time.perf_counter()
            B.celes_precond_build(ctx, edge)
            tb = time.perf_counter() - t0
            ip = B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_MIXED, use_precond=True)
            pre[f"edge_{int(edge)}nm"] = {"build_s": tb, "solve_s": ip["seconds"], "total_s": tb + ip["seconds"],
                                          "iterations": ip["iterations"], "residual": ip["residual"]}
        tt["block_preconditioned"] = pre
    if not args.no_plain:
        # (a) full size: plain FP64 GMRES for a bounded number of iterations
        #     gives its time per iteration; the time to 1e-6 is extrapolated
        #     with the iteration count the chosen form needed (labelled as such)
        cap = 24
        info_p = B.celes_solve(ctx, TOL, mode=B.CELES_SOLVE_FP64, max_iter=cap, use_precond=False,
                                raise_on_noconv=False)
        per_it = info_p["seconds"] / max(1, info_p["iterations"])
        tt["plain_fp64_s_per_iteration"] = per_it
        tt["plain_fp64_s_extrapolated"] = per_it * tt["chosen_iterations"]
        tt["speedup_extrapolated"] = tt["plain_fp64_s_extrapolated"] / tt["chosen_s"]
        tt["extrapolation"] = (f"plain FP64 GMRES timed for {info_p['iterations']} iterations at full size, "
                               f"times the {tt['chosen_iterations']} iterations of the chosen form")
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
            tt["measured_small"] = {"N": small.N, "chosen_s": im["seconds"], "chosen_iterations": im["iterations"],
                                    "plain_fp64_s": ip["seconds"], "plain_fp64_iterations": ip["iterations"],
                                    "plain_fp64_residual": ip["residual"], "chosen_residual": im["residual"],
                                    "speedup": ip["seconds"] / im["seconds"],
                                    "chosen_vs_plain_rel_l2": float(np.linalg.norm(bm - bp) / np.linalg.norm(bp)),
                                    "bicgstab_mixed": {"s": ib["seconds"], "iterations": ib["iterations"],
                                                       "matvecs_fp32": ib["matvecs_fp32"],
                                                       "residual": ib["residual"],
                                                       "vs_plain_rel_l2": float(np.linalg.norm(bb - bp) /
                                                                                np.linalg.norm(bp))}}
        finally:
            B.celes_destroy(cs)
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
        cores = host_cores()
        rows = args.cpu_rows or 24 * max(cores, 2)  # 10-20 s of oracle work
        sel = list(np.random.default_rng(7).choice(N, rows, replace=False))
        rate, dt = cpu_oracle_rate(scene, sel, cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{rows} receiver rows x {N - 1} sources of the oracle's FP64 on-the-fly coupling "
                         f"matvec (numpy, {cores} spawn workers), {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": workload_config(N, L, world),
                "roofline": roofline, "kernels": kernels, "time_to_1e-6": tt, "batched": batched, "learned_guess": learned,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
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
