"""Benchmark: one Newton linear solve of the condensed GL-DGSEM per step on GB300.

A step is one pass of the whole hot path on the 16^3-element, N = 4 Taylor-Green
workload (2,560,000 DOF, CFL 50): residual + Jacobian assembly, static condensation
(A_ii^-1, element Schur blocks, block-Jacobi factors), condensed right-hand side,
GMRES to a global relative residual of 1e-8, back-substitution.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--arm fp64|mixed|learned|batched] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 runs independent replicas (one per GPU); the
path has no collective.  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import sc_inputs as I  # noqa: E402

WORKLOAD = dict(name="tgv_16x16x16_N4_cfl50", n=16, N=4, Ma=0.1, Re=1600.0, cfl=50.0, seed=0, adv_flux=0,
                visc_flux=0)
METRIC = "linear-solve DOF/s at rel. residual 1e-8: condensed GPU forms vs plain FP64"
REL_TOL = 1e-8
# Peaks: HBM and bf16 from MEASURED_PEAKS.json; FP64 and FP32 FMA rates derived from
# the unit counts and clocks (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.26 TFLOP/s;
# a DFMA microbenchmark measured 1.20 TFLOP/s on this machine).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "_fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(device)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush(); self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def gather_max(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def train_correction(args, stream, cfl=None):
    """The learned arm's network, trained before the timed region on systems the method
    forms on the workload's own mesh and order (its element size and time step set the local
    physics the features see): Taylor-Green states of seeds 100.. (the timed system is seed 0)
    at Ma 0.05, 0.1 and 0.2, each with the CFL rule's time step at that Mach number; features
    and targets (the node blocks of the face-block inverses) of every boundary node from the
    library, shuffled mini-batch Adam through its kernels."""
    import torch
    from paper_1911_02366_gb300 import sc
    rng = np.random.default_rng(0)
    Fs, Ts = [], []
    t0 = time.perf_counter()
    n, N = WORKLOAD["n"], WORKLOAD["N"]
    cfl = WORKLOAD["cfl"] if cfl is None else cfl
    mach = (0.05, 0.1, 0.2)
    for i, Ma in enumerate(mach):
        Q, dt = I.tgv_state(n, N, Ma=Ma, seed=100 + i, cfl=cfl)
        c = sc.Context(stream=stream.cuda_stream, precision=sc.SC_PREC_MIXED, Ma=Ma, Re=WORKLOAD["Re"],
                       adv_flux=WORKLOAD["adv_flux"], visc_flux=WORKLOAD["visc_flux"],
                       precond=sc.SC_PC_RED_BLACK)
        c.sc_set_mesh(n, 2 * math.pi, N)
        c.sc_set_timestep(dt, 1)
        Qd = torch.tensor(Q.reshape(-1), device="cuda")
        c.sc_set_state(Qd, Qd)
        c.sc_assemble()
        c.sc_condense()
        K, _, _, nb = c.sc_sizes()
        nsmp = K * nb // 5
        F = torch.empty(nsmp, 128, device="cuda")
        sn = torch.empty(nsmp, device="cuda")
        T = torch.empty(nsmp, 25, device="cuda")
        c.sc_learned_features(F, sn)
        c.sc_learned_targets(T)
        Fs.append(F)
        Ts.append(T)
        c.close()
    X = torch.cat(Fs).contiguous()
    Y = torch.cat(Ts).contiguous()
    del Fs, Ts
    P = [rng.standard_normal((256, 128)) * math.sqrt(2 / 128), rng.standard_normal((256, 256)) * math.sqrt(2 / 256),
         rng.standard_normal((25, 256)) * math.sqrt(1 / 256) * 0.1]
    net = sc.MLP(np.concatenate([w.ravel() for w in P]), np.zeros(sc.MLP_NB), stream=stream.cuda_stream)
    hist = net.train(X, Y, epochs=args.train_epochs, batch=256, lr=1e-3)
    return net, {"samples": int(X.shape[0]), "systems": len(mach), "mesh": f"{n}^3 N={N}",
                 "epochs": args.train_epochs, "loss_first": hist[0], "loss_last": hist[-1],
                 "seconds": time.perf_counter() - t0}


def run_ours(args, world, rank, local):
    import torch
    from paper_1911_02366_gb300 import sc

    torch.cuda.set_device(local)
    W = WORKLOAD
    Q, dt = I.tgv_state(W["n"], W["N"], Ma=W["Ma"], seed=W["seed"], cfl=W["cfl"])
    dofs = Q.size
    precision = sc.SC_PREC_FP64 if args.arm == "fp64" else sc.SC_PREC_MIXED
    stream = torch.cuda.current_stream()
    extra = {}
    train_info = None
    if args.arm == "learned":
        net, train_info = train_correction(args, stream)
        extra = dict(precond=sc.SC_PC_LEARNED)
        if args.learned_min_reduction is not None:
            extra["learned_min_reduction"] = args.learned_min_reduction
    elif args.precond == "rb":
        extra = dict(precond=sc.SC_PC_RED_BLACK)
    elif args.precond == "rbs":
        extra = dict(precond=sc.SC_PC_RB_SCHUR if precision == sc.SC_PREC_MIXED else sc.SC_PC_RED_BLACK)
    ctx = sc.Context(stream=stream.cuda_stream, precision=precision, Re=W["Re"], Ma=W["Ma"],
                     adv_flux=W["adv_flux"], visc_flux=W["visc_flux"],
                     gmres_restart=args.restart, gmres_max_iters=args.max_iters, rel_tol=REL_TOL,
                     inner_tol=args.inner_tol, max_refine=20, tensor_cores=args.tensor_cores,
                     outer_krylov=args.outer_krylov if args.arm != "fp64" else 0, inner_iters=args.inner_iters,
                     explicit_schur=1 if args.operator == "explicit" else 0,
                     interior_fp64=args.interior_fp64 if args.arm != "fp64" else 0, **extra)

    ctx.sc_set_mesh(W["n"], 2 * math.pi, W["N"])
    if args.arm == "learned":
        ctx.sc_set_learned_weights(net)
    ctx.sc_set_timestep(dt, 1)
    Qd = torch.tensor(Q.reshape(-1), device="cuda")
    dQ = torch.zeros_like(Qd)
    ctx.sc_set_state(Qd, Qd)

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        ctx.sc_assemble()
        ev[1].record(stream)
        ctx.sc_condense()
        st = ctx.sc_solve(dQ, raise_on_not_converged=not args.allow_unconverged)
        ev[2].record(stream)
        return ev, st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    dominant = {"lu_solve": sc.SC_KERNEL_LU_SOLVE, "cond_boundary": sc.SC_KERNEL_COND_BOUNDARY,
                "cond_interior": sc.SC_KERNEL_COND_INTERIOR}[args.roofline_kernel]
    if args.operator == "explicit":
        dominant = sc.SC_KERNEL_EXPLICIT_APPLY
    ctx.sc_profile_kernel(dominant)
    sampler = ClockSampler(local) if rank == 0 else None
    l0 = ctx.sc_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True); end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    marks, stats = [], []
    for _ in range(args.steps):
        ev, st = step()
        marks.append(ev); stats.append(st)
    end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = ctx.sc_launch_count() - l0
    clocks = sampler.stop() if sampler else None
    total_ms = start.elapsed_time(end)
    assemble_ms = sum(ev[0].elapsed_time(ev[1]) for ev in marks)
    solve_ms = sum(ev[1].elapsed_time(ev[2]) for ev in marks)
    n_prof, prof_ms = ctx.sc_profile_read()
    prof_elems = ctx.sc_profile_elements()
    ctx.sc_profile_kernel(-1)
    total_ms = gather_max(world, total_ms)
    worst = max(s["rel_residual"] for s in stats)
    ok = all(s["status"] == 0 for s in stats) and worst <= REL_TOL

    # end to end: host (pinned) state in, host update out, inside the timed region
    Qh = torch.tensor(Q.reshape(-1)).pin_memory()
    dQh = torch.zeros(dofs, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.sc_set_state(Qh, Qh)
        ctx.sc_assemble()
        ctx.sc_condense()
        ctx.sc_solve(dQh, raise_on_not_converged=not args.allow_unconverged)
    torch.cuda.synchronize()
    e2e_s = gather_max(world, time.perf_counter() - t0)

    flops, bytes_ = ctx.sc_kernel_work(dominant)  # a launch over all K elements
    K_all = ctx.sc_sizes()[0]
    per_launch = prof_elems / max(n_prof, 1)  # the red-black sweep's launches cover one colour
    flops, bytes_ = flops * per_launch / K_all, bytes_ * per_launch / K_all
    avg_ms = prof_ms / max(n_prof, 1)
    peaks = measured_peaks()
    if args.arm == "fp64":
        roof = {"bound": "alu", "achieved": flops / (avg_ms * 1e-3) / 1e12,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s"}
    else:
        roof = {"bound": "hbm", "achieved": bytes_ / (avg_ms * 1e-3) / 1e9,
                "peak": float(peaks["hbm_gbs"]), "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = (TRAFFIC.get((args.arm, dominant)) * per_launch / K_all
                       if (W["n"], W["N"]) == (16, 4) and args.precond in ("rb", "rbs") and args.arm == "mixed"
                       and TRAFFIC.get((args.arm, dominant)) else None)
    roof["kernel"] = {sc.SC_KERNEL_LU_SOLVE: "k_lu_solve", sc.SC_KERNEL_COND_BOUNDARY: "k_cond_boundary_pk",
                      sc.SC_KERNEL_COND_INTERIOR: "k_cond_interior_pk",
                      sc.SC_KERNEL_EXPLICIT_APPLY: "k_explicit_w"}[dominant]
    roof["launches_timed"] = n_prof
    roof["avg_launch_ms"] = avg_ms
    roof["elements_per_launch"] = per_launch

    value = world * dofs * args.steps / (total_ms * 1e-3)
    K_, ne_, ni_, nb_ = ctx.sc_sizes()
    lda_ = ((((ni_ + 3) // 4) * 4 + nb_ + 3) // 4) * 4
    blocks_gb = K_ * ne_ * lda_ * 8 / 1e9  # the assembled FP64 own blocks
    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.arm == "fp64" else "f32+f64",
        "data": "synthetic (seeded Taylor-Green state, 1e-3 perturbation)",
        "config": {"workload": W["name"], "elements": W["n"] ** 3, "order": W["N"], "dof": dofs, "cfl": W["cfl"],
                   "Ma": W["Ma"], "Re": W["Re"], "arm": args.arm, "gmres_restart": args.restart,
                   "fluxes": ("lax-friedrichs" if W["adv_flux"] else "roe") + " + "
                   + ("sipg" if W["visc_flux"] else "br1"),
                   "inner_tol": args.inner_tol if args.arm != "fp64" else None,
                   "outer": (f"fgmres({args.outer_krylov})" if args.outer_krylov else "refinement sweeps")
                   if args.arm != "fp64" else None,
                   "tensor_cores": bool(args.tensor_cores) if args.arm != "fp64" else False,
                   "operator": args.operator, "precond": "learned" if args.arm == "learned" else args.precond,
                   "l2": f"inputs larger than L2 (element blocks {blocks_gb:.1f} GB)", "parallelism": f"replicas x{world}"},
        "linear_solve_dof_per_s": world * dofs * args.steps / (gather_max(world, solve_ms) * 1e-3),
        "assemble_ms_per_step": assemble_ms / args.steps,
        "gmres_iters": [s["gmres_iters"] for s in stats],
        "learned_fallbacks": [s["learned_fallbacks"] for s in stats] if args.arm == "learned" else None,
        "training": train_info,
        "refinement_sweeps": [s["refinements"] for s in stats],
        "rel_residual_max": worst, "converged": ok,
        "e2e": {"value": world * dofs * e2e_steps / e2e_s, "unit": "DOF/s",
                "h2d_bytes_per_step": 2 * dofs * 8, "d2h_bytes_per_step": dofs * 8},
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clocks,
    }
    if args.arm != "fp64" and not args.no_fp64_arm:
        line["fp64_arm"] = fp64_reference_arm(args, W, Q, dt, stream, dQ)
        line["speedup_vs_fp64_arm"] = value / line["fp64_arm"]["value"]
    ctx.close()
    return line


def fp64_reference_arm(args, W, Q, dt, stream, dQ_mixed):
    """The metric's denominator in the same run: the plain FP64 condensed GPU solve (FP64
    blocks and operator, block-Jacobi GMRES(30), no refinement) of the same system, timed the
    same way (2 timed steps after 1 warm-up); and the relative difference of the two arms'
    solutions (the FP64 arm matches the oracle's global solve to 1e-10 on the 4^3, N = 3
    system in the tests)."""
    import torch
    from paper_1911_02366_gb300 import sc
    ctx = sc.Context(stream=stream.cuda_stream, precision=sc.SC_PREC_FP64, Re=W["Re"], Ma=W["Ma"],
                     adv_flux=W["adv_flux"], visc_flux=W["visc_flux"],
                     gmres_restart=30, gmres_max_iters=args.max_iters, rel_tol=REL_TOL)
    ctx.sc_set_mesh(W["n"], 2 * math.pi, W["N"])
    ctx.sc_set_timestep(dt, 1)
    Qd = torch.tensor(Q.reshape(-1), device="cuda")
    dQ = torch.zeros_like(Qd)
    ctx.sc_set_state(Qd, Qd)

    def step():
        ctx.sc_assemble()
        ctx.sc_condense()
        return ctx.sc_solve(dQ)

    step()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    stats = [step() for _ in range(2)]
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 2
    diff = float(torch.linalg.vector_norm(dQ_mixed - dQ) / torch.linalg.vector_norm(dQ))
    ctx.close()
    return {"value": Q.size / (ms * 1e-3), "unit": "DOF/s", "ms_per_step": ms, "steps": 2, "warmup": 1,
            "precond": "bj", "gmres_iters": [s["gmres_iters"] for s in stats],
            "rel_residual_max": max(s["rel_residual"] for s in stats),
            "solution_rel_diff_mixed_vs_fp64": diff}


# DRAM traffic per launch over all elements (dram__bytes_read.sum + dram__bytes_write.sum)
# from the one-pass ncu capture of the bench workload summarised in profiles/; None for the
# kernels changed since.
TRAFFIC = {
    # k_lu_solve<float, float, 1> on one colour (2048 elements) of the 16^3, N = 4 workload:
    # 2,043,262,464 + 93,952 bytes; x2 for a launch over all 4096 elements
    # (profiles/dram_traffic_tgv_16x16x16_N4_rb_schur.md)
    ("mixed", 2): 2 * (2043262464 + 93952),
}


def cpu_sample(seed=0):
    """Bounded sample of the workload for the oracle: the periodic Taylor-Green box on
    3^3 elements at the same order N = 4 and the same time step as the 16^3 workload
    (same per-element blocks and physics, 27 instead of 4096 elements)."""
    W = WORKLOAD
    n_s = 3
    _, dt = I.tgv_state(W["n"], W["N"], Ma=W["Ma"], seed=W["seed"], cfl=W["cfl"])
    Q, _ = I.tgv_state(n_s, W["N"], Ma=W["Ma"], seed=seed, cfl=W["cfl"])
    return n_s, 2 * math.pi, Q, dt


def run_oracle(steps: int):
    """The FP64 CPU oracle's condensed linear solve (condensation, block-Jacobi GMRES(30),
    back-substitution) on the bounded sample; the Jacobian is assembled beforehand."""
    import oracle as O
    n_s, L, Q, dt = cpu_sample()
    W = WORKLOAD
    p = O.Params(n=n_s, N=W["N"], dt=dt, L=L, Re=W["Re"], Ma=W["Ma"], adv_flux=W["adv_flux"],
                 visc_flux=W["visc_flux"])
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    times, iters = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        x, info = O.condensed_solve(A, B, n_s, W["N"], method="gmres", tol=REL_TOL, restart=30, maxiter=5000)
        times.append(time.perf_counter() - t0)
        iters.append(info.get("iters"))
    res = float(np.linalg.norm(B - A @ x) / np.linalg.norm(B))
    return {"dof": Q.size, "seconds": times, "iters": iters, "rel_residual": res,
            "sample": f"periodic Taylor-Green box on {n_s}^3 elements, N={W['N']}, dt of the 16^3 workload; "
                      "one linear solve (condense, GMRES(30) to 1e-8, back-substitute), Jacobian assembled beforehand"}


BATCH_ORDERS = ((7, 2), (7, 3), (7, 4), (7, 5), (7, 6))  # (elements per direction, N) of the uneven-order batch
BATCH_CFL = 10.0  # GMRES(30) stalls on these small meshes at CFL 50


def run_batched(args, world, rank, local):
    """Uneven-order batch: one system per order N = 2..6 on 7^3 elements each (1715
    elements, the size of a 12^3 mesh with N drawn uniformly from 2..6, each order as its
    own conforming system).  A step assembles every system, condenses all of them in one
    replayed CUDA graph (grouped launches, autotuned TF32 tiles) and solves each to 1e-8."""
    import torch
    from paper_1911_02366_gb300 import sc

    torch.cuda.set_device(local)
    W = WORKLOAD
    stream = torch.cuda.current_stream()
    ctxs, states, dofs = [], [], 0
    for n, N in BATCH_ORDERS:
        Q, dt = I.tgv_state(n, N, Ma=W["Ma"], seed=W["seed"], cfl=BATCH_CFL)
        c = sc.Context(stream=stream.cuda_stream, precision=sc.SC_PREC_MIXED, Re=W["Re"], Ma=W["Ma"],
                       adv_flux=W["adv_flux"], visc_flux=W["visc_flux"],
                       gmres_restart=args.restart, gmres_max_iters=args.max_iters, rel_tol=REL_TOL,
                       inner_tol=args.inner_tol, max_refine=20)
        c.sc_set_mesh(n, 2 * math.pi, N)
        c.sc_set_timestep(dt, 1)
        Qd = torch.tensor(Q.reshape(-1), device="cuda")
        c.sc_set_state(Qd, Qd)
        ctxs.append(c)
        states.append((Qd, torch.zeros_like(Qd)))
        dofs += Q.size
    batch = sc.Batch(ctxs)

    def step(batched=True):
        for c in ctxs:
            c.sc_assemble()
        if batched:
            batch.condense(graph=True, autotune=True)
        else:
            for c in ctxs:
                c.sc_condense()
        return [c.sc_solve(dq, raise_on_not_converged=not args.allow_unconverged) for c, (_, dq) in zip(ctxs, states)]

    def condense_ms(batched, reps=3):
        for c in ctxs:
            c.sc_assemble()
        t0 = torch.cuda.Event(enable_timing=True); t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            if batched:
                batch.condense(graph=True, autotune=True)
            else:
                for c in ctxs:
                    c.sc_condense()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / reps

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    big = ctxs[-1]
    big.sc_profile_kernel(sc.SC_KERNEL_LU_SOLVE)
    sampler = ClockSampler(local) if rank == 0 else None
    l0 = sum(c.sc_launch_count() for c in ctxs)
    barrier(world)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True); end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step())
    end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = sum(c.sc_launch_count() for c in ctxs) - l0
    clocks = sampler.stop() if sampler else None
    n_prof, prof_ms = big.sc_profile_read()
    big.sc_profile_kernel(-1)
    total_ms = gather_max(world, start.elapsed_time(end))
    worst = max(s["rel_residual"] for st in stats for s in st)
    ms_batched = condense_ms(True)
    ms_separate = condense_ms(False)

    # end to end: host (pinned) states in, host updates out
    hosts = [(torch.tensor(Qd.cpu().numpy()).pin_memory(), torch.zeros(Qd.numel(), dtype=torch.float64).pin_memory())
             for Qd, _ in states]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for c, (qh, _) in zip(ctxs, hosts):
            c.sc_set_state(qh, qh)
            c.sc_assemble()
        batch.condense(graph=True, autotune=True)
        for c, (_, dqh) in zip(ctxs, hosts):
            c.sc_solve(dqh, raise_on_not_converged=not args.allow_unconverged)
    torch.cuda.synchronize()
    e2e_s = gather_max(world, time.perf_counter() - t0)

    flops, bytes_ = big.sc_kernel_work(sc.SC_KERNEL_LU_SOLVE)
    avg_ms = prof_ms / max(n_prof, 1)
    peaks = measured_peaks()
    roof = {"bound": "hbm", "achieved": bytes_ / (avg_ms * 1e-3) / 1e9, "peak": float(peaks["hbm_gbs"]),
            "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof.update(traffic=None, kernel=f"k_lu_solve (N = {BATCH_ORDERS[-1][1]} system)", launches_timed=n_prof,
                avg_launch_ms=avg_ms)
    tiles = {f"ni={t[0]}": {"Y": t[1], "S": t[2], "LU": t[3]}
             for t in (batch.tiles(i) for i in range(len(BATCH_ORDERS)))}
    line = {
        "metric": METRIC, "value": world * dofs * args.steps / (total_ms * 1e-3), "unit": "DOF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded Taylor-Green states, 1e-3 perturbation)",
        "config": {"workload": "tgv_uneven_order_7x7x7_N2_to_N6_cfl10", "systems": [list(o) for o in BATCH_ORDERS],
                   "elements": sum(n ** 3 for n, _ in BATCH_ORDERS), "dof": dofs, "cfl": BATCH_CFL,
                   "arm": "batched", "gmres_restart": args.restart, "inner_tol": args.inner_tol,
                   "l2": "inputs larger than L2 (element blocks of the N = 5, 6 systems alone exceed it)",
                   "parallelism": f"replicas x{world}"},
        "condense_ms_batched_graph": ms_batched, "condense_ms_separate": ms_separate, "autotuned_tiles": tiles,
        "gmres_iters": [[s["gmres_iters"] for s in st] for st in stats], "rel_residual_max": worst,
        "converged": worst <= REL_TOL,
        "e2e": {"value": world * dofs * e2e_steps / e2e_s, "unit": "DOF/s", "h2d_bytes_per_step": 2 * dofs * 8,
                "d2h_bytes_per_step": dofs * 8},
        "gpu_launches": launches, "roofline": roof, "clocks": clocks,
    }
    batch.close()
    for c in ctxs:
        c.close()
    return line


MIXED_MESH = dict(n=12, order_seed=1, cfl=10.0)  # 12^3 elements, N drawn uniformly from 2..6


def run_mixed_mesh(args, world, rank, local):
    """One 12^3 mesh whose element orders are drawn uniformly from 2..6 (seed 1), mortar faces
    between orders.  A step sets the state, condenses (element blocks by dual numbers, grouped
    condensation of all orders at once) and solves A dQ = -R to 1e-8 (FP32 condensed GMRES,
    S through Jacobian-vector products, FP64 refinement)."""
    import torch
    from paper_1911_02366_gb300 import sc

    torch.cuda.set_device(local)
    W = WORKLOAD
    n = args.n or MIXED_MESH["n"]
    orders = I.order_draw(MIXED_MESH["order_seed"], n ** 3)
    Q, dt = I.tgv_state_mixed(n, orders, Ma=W["Ma"], seed=W["seed"], cfl=MIXED_MESH["cfl"])
    Q = np.ascontiguousarray(Q.reshape(-1))
    dofs = Q.size
    stream = torch.cuda.current_stream()
    ctx = sc.MixedContext(n, orders, 2 * math.pi, stream=stream.cuda_stream, Re=W["Re"], Ma=W["Ma"],
                          adv_flux=W["adv_flux"], gmres_restart=args.restart, gmres_max_iters=args.max_iters,
                          rel_tol=REL_TOL, inner_tol=args.inner_tol, max_refine=20)
    Qd = torch.tensor(Q, device="cuda")
    dQ = torch.zeros_like(Qd)
    split = {"condense": 0.0, "solve": 0.0}

    def step(timed=False):
        ctx.set_state(Qd, Qd, dt=dt)
        t0 = time.perf_counter()
        ctx.condense()
        t1 = time.perf_counter()
        st = ctx.solve(dQ, raise_on_not_converged=not args.allow_unconverged)
        if timed:
            split["condense"] += t1 - t0
            split["solve"] += time.perf_counter() - t1
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if rank == 0 else None
    l0 = ctx.launch_count()
    ctx.profile(True)
    barrier(world)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True); end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    stats = [step(timed=True) for _ in range(args.steps)]
    end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = ctx.launch_count() - l0
    n_apps, apps_ms, app_bytes = ctx.profile_read()
    ctx.profile(False)
    peaks = measured_peaks()
    avg_ms = apps_ms / max(n_apps, 1)
    roof = {"bound": "hbm", "achieved": app_bytes / (avg_ms * 1e-3) / 1e9, "peak": float(peaks["hbm_gbs"]),
            "unit": "GB/s", "traffic": None,
            "kernel": "block-Jacobi application (k_lu_solve_cta, one launch per order class, concurrent)",
            "launches_timed": n_apps, "avg_launch_ms": avg_ms}
    roof["frac"] = roof["achieved"] / roof["peak"]
    clocks = sampler.stop() if sampler else None
    total_ms = gather_max(world, start.elapsed_time(end))
    worst = max(s["rel_residual"] for s in stats)
    # end to end: pinned host state in, host update out
    qh = torch.tensor(Q).pin_memory()
    dqh = torch.zeros(dofs, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.set_state(qh, qh, dt=dt)
        ctx.condense()
        ctx.solve(dqh, raise_on_not_converged=not args.allow_unconverged)
    torch.cuda.synchronize()
    e2e_s = gather_max(world, time.perf_counter() - t0)
    counts = {int(N): int((orders == N).sum()) for N in range(2, 7)}
    line = {
        "metric": METRIC, "value": world * dofs * args.steps / (total_ms * 1e-3), "unit": "DOF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded Taylor-Green state on a mixed-order mesh, 1e-3 perturbation)",
        "config": {"workload": f"tgv_{n}x{n}x{n}_N2_to_N6_drawn_cfl{MIXED_MESH['cfl']:g}", "elements": n ** 3,
                   "orders": counts, "dof": dofs, "cfl": MIXED_MESH["cfl"], "arm": "mixedmesh",
                   "gmres_restart": args.restart, "inner_tol": args.inner_tol, "fluxes": "roe + br1, mortar faces",
                   "l2": "inputs larger than L2 (FP32 element blocks)", "parallelism": f"replicas x{world}"},
        "condense_ms_per_step": 1e3 * split["condense"] / args.steps,
        "solve_ms_per_step": 1e3 * split["solve"] / args.steps,
        "gmres_iters": [s["gmres_iters"] for s in stats], "refinement_sweeps": [s["refinements"] for s in stats],
        "rel_residual_max": worst, "converged": worst <= REL_TOL,
        "e2e": {"value": world * dofs * e2e_steps / e2e_s, "unit": "DOF/s", "h2d_bytes_per_step": 2 * dofs * 8,
                "d2h_bytes_per_step": dofs * 8},
        "gpu_launches": launches, "roofline": roof, "clocks": clocks,
    }
    ctx.close()
    return line


def cpu_threads():
    try:
        import oracle as O
        return O.num_threads()
    except Exception:
        return os.cpu_count()


def run_timesteps(args, world, rank, local):
    """Implicit time stepping of the workload's state: BDF2 steps (the first BDF1) at the
    given CFL, each solved by Newton iterations (sc_newton_step: assemble, condense, solve,
    update) until ||R|| <= newton_tol ||R_0||.  The value is DOF x time steps per second of
    the whole loop; the per-step Newton and GMRES counts go with it."""
    import torch
    from paper_1911_02366_gb300 import sc

    torch.cuda.set_device(local)
    W = WORKLOAD
    Q, dt = I.tgv_state(W["n"], W["N"], Ma=W["Ma"], seed=W["seed"], cfl=args.cfl)
    dofs = Q.size
    stream = torch.cuda.current_stream()
    pc = {"bj": sc.SC_PC_BLOCK_JACOBI, "rb": sc.SC_PC_RED_BLACK, "rbs": sc.SC_PC_RB_SCHUR,
          "learned": sc.SC_PC_LEARNED}[args.ts_precond]
    net, train_info = (train_correction(args, stream, cfl=args.cfl) if pc == sc.SC_PC_LEARNED else (None, None))
    ctx = sc.Context(stream=stream.cuda_stream, precision=sc.SC_PREC_MIXED, Re=W["Re"], Ma=W["Ma"],
                     adv_flux=W["adv_flux"], visc_flux=W["visc_flux"],
                     gmres_restart=args.restart, gmres_max_iters=args.max_iters, rel_tol=REL_TOL,
                     inner_tol=args.inner_tol, max_refine=20, tensor_cores=args.tensor_cores,
                     outer_krylov=args.outer_krylov, inner_iters=args.inner_iters, precond=pc,
                     interior_fp64=args.interior_fp64)
    ctx.sc_set_mesh(W["n"], 2 * math.pi, W["N"])
    if net is not None:
        ctx.sc_set_learned_weights(net)
    Qs = torch.tensor(Q.reshape(-1), device="cuda")
    Qsm1 = None
    sampler = ClockSampler(local) if rank == 0 else None
    l0 = ctx.sc_launch_count()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True); end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    steps = []
    failure = None
    for s in range(args.time_steps):
        bdf = 1 if Qsm1 is None else 2
        ctx.sc_set_timestep(dt, bdf)
        ctx.sc_set_state(Qs, Qs, Qsm1)  # Newton starts from the last level
        try:
            it, nrel, st = ctx.sc_newton_step(max_newton=args.max_newton, newton_tol=args.newton_tol)
        except sc.SCError as ex:  # recorded with the steps done so far; the line says it did not finish
            failure = {"step": s, "bdf": bdf, "error": str(ex)}
            break
        Qn = torch.empty_like(Qs)
        ctx.sc_get_state(Qn)
        Qsm1, Qs = Qs, Qn
        steps.append({"bdf": bdf, "newton": it, "newton_rel": nrel, "last_gmres_iters": st["gmres_iters"],
                      "last_rel_residual": st["rel_residual"], "last_learned_fallbacks": st["learned_fallbacks"]})
    end.record(stream)
    torch.cuda.synchronize()
    launches = ctx.sc_launch_count() - l0
    clocks = sampler.stop() if sampler else None
    total_ms = gather_max(world, start.elapsed_time(end))
    ctx.close()
    return {
        "metric": "implicit time steps: DOF x steps / s (Newton on each step, condensed mixed-precision solves)",
        "value": world * dofs * len(steps) / (total_ms * 1e-3), "unit": "DOF*steps/s", "n_gpus": world,
        "steps": args.time_steps, "warmup": 0, "ms_per_step": total_ms / max(len(steps), 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded Taylor-Green state, 1e-3 perturbation)",
        "config": {"workload": f"tgv_{W['n']}x{W['n']}x{W['n']}_N{W['N']}_bdf2_cfl{args.cfl:g}",
                   "elements": W["n"] ** 3, "order": W["N"], "dof": dofs, "cfl": args.cfl, "dt": dt,
                   "newton_tol": args.newton_tol, "linear_rel_tol": REL_TOL, "arm": "timesteps",
                   "outer": f"fgmres({args.outer_krylov})" if args.outer_krylov else "refinement sweeps",
                   "inner_iters_cap": args.inner_iters or None, "precond": args.ts_precond,
                   "interior_fp64": bool(args.interior_fp64),
                   "gmres_restart": args.restart, "parallelism": f"replicas x{world}"},
        "training": train_info,
        "time_steps": steps, "newton_total": sum(x["newton"] for x in steps),
        "completed_steps": len(steps), "failure": failure,
        "gpu_launches": launches, "clocks": clocks,
    }


def eta(res, ms, decades=1.0):
    """Convergence rate of Sec. 4: the slope of log10 ||M^-1 H||_inf against the compute time
    (1/s) over the final `decades` of the history."""
    res, ms = np.asarray(res, float), np.asarray(ms, float)
    ok = np.isfinite(res) & (res > 0)
    res, ms = res[ok], ms[ok]
    if len(res) < 2:
        return None
    sel = np.log10(res) <= np.log10(res[-1]) + decades
    if sel.sum() < 2:
        sel[-2:] = True
    t, y = ms[sel] * 1e-3, np.log10(res[sel])
    if t.max() <= t.min():
        return None
    return float(np.polyfit(t, y, 1)[0])


def run_march(args, world, rank, local):
    """The paper's steady-state experiment (Sec. 4) restated on a decaying Taylor-Green state:
    explicit low-storage RK3 against frozen-Jacobian BDF1 solved globally (dense LU of A) and
    by static condensation (dense LU of S, and the condensed GMRES), each to
    ||M^-1 H||_inf <= steady_tol; time to the tolerance, eta, and the one-time and per-step
    costs of Tables tab:SpeedUp, tab:Advantages and tab:Advantages2."""
    import torch
    from paper_1911_02366_gb300 import sc

    torch.cuda.set_device(local)
    n, N = args.n or 4, args.order or 3
    Ma, Re = args.march_ma, args.march_re
    Q, _ = I.tgv_state(n, N, Ma=Ma, seed=0, cfl=1.0)
    dofs = Q.size
    stream = torch.cuda.current_stream()
    prec = sc.SC_PREC_FP64 if args.march_precision == "fp64" else sc.SC_PREC_MIXED

    def ctx_new(**kw):
        c = sc.Context(stream=stream.cuda_stream, precision=prec, Re=Re, Ma=Ma, rel_tol=1e-10,
                       gmres_restart=args.restart, gmres_max_iters=args.max_iters, max_refine=40,
                       tensor_cores=args.tensor_cores, **kw)
        c.sc_set_mesh(n, 2 * math.pi, N)
        Qd = torch.tensor(Q.reshape(-1), device="cuda")
        c.sc_set_state(Qd, Qd)
        return c

    out = {}
    tol = args.steady_tol
    # explicit RK3 in chunks until the tolerance or the step cap
    c = ctx_new()
    res_all, t_all, t0, steps = [c.sc_steady_residual()], [0.0], 0.0, 0
    while res_all[-1] > tol and steps < args.max_explicit_steps:
        k = min(2000, args.max_explicit_steps - steps)
        res, dts, ms = c.sc_explicit_march(args.explicit_cfl, k, dfl=args.explicit_dfl)
        res_all += list(res[1:])
        t_all += list(t0 + ms * np.arange(1, k + 1) / k)
        t0 += ms
        steps += k
    hit = next((i for i, r in enumerate(res_all) if r <= tol), None)
    out["explicit_rk3"] = {"steps": hit if hit is not None else steps, "reached": hit is not None,
                           "seconds_to_tol": (t_all[hit] if hit is not None else t0) * 1e-3,
                           "final_residual": res_all[-1], "eta_per_s": eta(res_all, t_all),
                           "cfl": args.explicit_cfl}
    c.close()
    # implicit BDF1 with a frozen Jacobian, three solvers
    for name, direct, extra in (("bdf1_global_lu", "A", {}), ("bdf1_condensed_lu", "S", {}),
                                ("bdf1_condensed_gmres", None, {"precond": sc.SC_PC_RED_BLACK})):
        c = ctx_new(**extra)
        res, ms, its = c.sc_implicit_march(args.march_dt, args.max_implicit_steps, jacobian_every=0, direct=direct,
                                           steady_tol=tol)
        hit = next((i for i, r in enumerate(res) if r <= tol), None)
        row = {"steps": hit if hit is not None else len(res) - 1, "reached": hit is not None,
               "seconds_to_tol": (ms[hit] if hit is not None else ms[-1]) * 1e-3, "final_residual": float(res[-1]),
               "eta_per_s": eta(res[:hit + 1] if hit else res, ms[:hit + 1] if hit else ms),
               "first_step_ms": float(ms[1]), "later_step_ms": float(np.median(np.diff(ms[1:]))) if len(ms) > 2 else None}
        if direct is None:
            row["gmres_iters_per_step"] = float(np.mean(its))
        c.close()
        # one-time and per-solve costs (Tables tab:Advantages, tab:Advantages2)
        if direct is not None:
            c = ctx_new()
            c.sc_set_timestep(args.march_dt, 1)
            c.sc_assemble()
            c.sc_condense()
            form_ms, fac_ms = c.sc_direct_factor(direct)
            dQ = torch.zeros(dofs, dtype=torch.float64, device="cuda")
            st = c.sc_direct_solve(dQ, raise_on_not_converged=False)
            row.update({"form_ms": form_ms, "lu_factor_ms": fac_ms, "lu_solve_ms_per_solve": st["ms_gmres"] / max(st["refinements"], 1),
                        "cond_ops_ms_per_solve": st["ms_rhs"] / max(st["refinements"], 1), "sweeps": st["refinements"]})
            c.close()
        out[name] = row
    g, cs = out["bdf1_global_lu"], out["bdf1_condensed_lu"]
    ex = out["explicit_rk3"]
    speed = {k: (ex["seconds_to_tol"] / v["seconds_to_tol"] if v["reached"] and ex["reached"] else None)
             for k, v in out.items() if k != "explicit_rk3"}
    return {
        "metric": "time to steady state ||M^-1 H||_inf <= tol (s): explicit RK3 vs frozen-Jacobian BDF1, global vs condensed",
        "value": cs["seconds_to_tol"], "unit": "s", "n_gpus": world, "steps": cs["steps"], "warmup": 0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == sc.SC_PREC_FP64 else "f32+f64", "data": "synthetic (decaying Taylor-Green state)",
        "config": {"workload": f"tgv_{n}x{n}x{n}_N{N}_Re{Re:g}_Ma{Ma:g}", "elements": n ** 3, "order": N, "dof": dofs,
                   "steady_tol": tol, "bdf1_dt": args.march_dt, "arm": "march", "precision": args.march_precision},
        "methods": out,
        "speedup_vs_explicit": speed,
        "eta_ratio_condensed_over_global": (cs["eta_per_s"] / g["eta_per_s"]
                                            if cs["eta_per_s"] and g["eta_per_s"] else None),
        "speedup_condensed_over_global": (g["seconds_to_tol"] / cs["seconds_to_tol"]
                                          if g["reached"] and cs["reached"] else None),
    }


def run_peaks(args, world, rank, local):
    """Peak rates of the arithmetic this project's kernels run in, on this GPU: dense GEMM
    through cuBLAS (torch.matmul) in FP64 and in TF32 (FP32 storage, TF32 tensor cores), and
    this library's TF32 tcgen05 GEMM (sc_gemm_tf32) at the same size; best of 5 after 2
    warm-ups, CUDA events."""
    import torch
    from paper_1911_02366_gb300 import sc
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()

    def best(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            a.record(stream); fn(); b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    out = {}
    n64 = 8192
    A = torch.randn(n64, n64, dtype=torch.float64, device="cuda")
    B = torch.randn(n64, n64, dtype=torch.float64, device="cuda")
    ms = best(lambda: torch.matmul(A, B))
    out["fp64_gemm_cublas_tflops"] = 2 * n64 ** 3 / (ms * 1e-3) / 1e12
    del A, B
    n32 = 8192
    A = torch.randn(n32, n32, dtype=torch.float32, device="cuda")
    B = torch.randn(n32, n32, dtype=torch.float32, device="cuda")
    C = torch.empty(n32, n32, dtype=torch.float32, device="cuda")
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    ms = best(lambda: torch.matmul(A, B, out=C))
    torch.backends.cuda.matmul.allow_tf32 = prev
    out["tf32_gemm_cublas_tflops"] = 2 * n32 ** 3 / (ms * 1e-3) / 1e12
    ms = best(lambda: sc.sc_gemm_tf32(A.view(1, n32, n32), B.view(1, n32, n32), C.view(1, n32, n32),
                                      stream=stream.cuda_stream))
    out["tf32_gemm_sc_tflops"] = 2 * n32 ** 3 / (ms * 1e-3) / 1e12
    peaks = measured_peaks()
    return {"metric": "peak rates of the arithmetic on this GPU (GEMM)", "value": out["tf32_gemm_sc_tflops"],
            "unit": "TFLOP/s", "n_gpus": world, "steps": 5, "warmup": 2, "higher_is_better": True,
            "config": {"workload": f"gemm {n32}^3 (TF32), {n64}^3 (FP64)", "arm": "peaks"},
            **out, "bf16_cublas_measured_tflops": peaks.get("bf16_tflops"), "hbm_measured_gbs": peaks.get("hbm_gbs")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--arm", choices=["fp64", "mixed", "learned", "batched", "mixedmesh", "timesteps", "march", "peaks"],
                    default="mixed")
    ap.add_argument("--steady-tol", type=float, default=1e-9, help="march arm: ||M^-1 H||_inf of the steady state")
    ap.add_argument("--march-dt", type=float, default=1.0, help="march arm: BDF1 time step (the paper's dt = 1)")
    ap.add_argument("--march-re", type=float, default=30.0, help="march arm: Reynolds number (the paper's 30)")
    ap.add_argument("--march-ma", type=float, default=0.2, help="march arm: Mach number (the paper's 0.2)")
    ap.add_argument("--march-precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--explicit-cfl", type=float, default=0.15, help="march arm: RK3 CFL (h/N spacing)")
    ap.add_argument("--explicit-dfl", type=float, default=0.5, help="march arm: RK3 diffusive limit factor")
    ap.add_argument("--max-explicit-steps", type=int, default=200000)
    ap.add_argument("--max-implicit-steps", type=int, default=400)
    ap.add_argument("--time-steps", type=int, default=10, help="timesteps arm: BDF2 steps")
    ap.add_argument("--cfl", type=float, default=100.0, help="timesteps arm: CFL of the time step")
    ap.add_argument("--ts-precond", choices=["bj", "rb", "rbs", "learned"], default="rb",
                    help="timesteps arm: preconditioner of the condensed GMRES (learned: trained first, untimed)")
    ap.add_argument("--newton-tol", type=float, default=1e-6, help="timesteps arm: ||R|| / ||R_0|| per step")
    ap.add_argument("--max-newton", type=int, default=8, help="timesteps arm: Newton updates per step")
    ap.add_argument("--train-epochs", type=int, default=8, help="learned arm: training epochs (untimed)")
    ap.add_argument("--learned-min-reduction", type=float, default=None,
                    help="learned arm: restart-cycle reduction below which the solve falls back to block Jacobi")
    ap.add_argument("--operator", choices=["implicit", "explicit"], default="implicit",
                    help="mixed arm: condensed operator applied implicitly or from explicit W_e blocks")
    ap.add_argument("--precond", choices=["bj", "rb", "rbs"], default="rbs",
                    help="condensed preconditioner: block Jacobi, the red-black block Gauss-Seidel sweep, or the "
                         "sweep with Schur-corrected black blocks (mixed arm; the FP64 arm takes the plain sweep)")
    ap.add_argument("--roofline-kernel", choices=["lu_solve", "cond_boundary", "cond_interior"], default="lu_solve",
                    help="the kernel whose launches the roofline object times (the step's largest share)")
    ap.add_argument("--interior-fp64", type=int, choices=[0, 1], default=0,
                    help="mixed arms, N >= 5: A_ii^-1 by FP64 Gauss-Jordan, rounded to FP32 for the operator")
    ap.add_argument("--adv-flux", choices=["roe", "lf"], default="roe",
                    help="advective numerical flux: Roe (default) or local Lax-Friedrichs (the paper's experiment)")
    ap.add_argument("--visc-flux", choices=["br1", "sipg"], default="br1",
                    help="viscous numerical flux: BR1 (default) or the symmetric interior penalty (the "
                         "paper's experiment; compact)")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--max-iters", type=int, default=4000)
    ap.add_argument("--inner-tol", type=float, default=1e-4)
    ap.add_argument("--outer-krylov", type=int, default=0,
                    help="mixed arms: 0 = refinement sweeps, m > 0 = outer FGMRES(m) on the FP64 system")
    ap.add_argument("--inner-iters", type=int, default=0, help="mixed arms: cap per inner condensed solve (0 = none)")
    ap.add_argument("--tensor-cores", type=int, choices=[0, 1], default=1,
                    help="mixed arm: TF32 tcgen05 Schur products and LU trailing updates (1) or FP32 CUDA cores (0)")
    ap.add_argument("--n", type=int, default=None, help="elements per direction (profiling runs)")
    ap.add_argument("--order", type=int, default=None, help="polynomial order (profiling runs)")
    ap.add_argument("--allow-unconverged", action="store_true", help="profiling runs with capped iterations")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true", help="skip the plain FP64 arm beside the mixed line")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.n or args.order:
        n = args.n or WORKLOAD["n"]; N = args.order or WORKLOAD["N"]
        WORKLOAD.update(n=n, N=N, name=f"tgv_{n}x{n}x{n}_N{N}_cfl{int(WORKLOAD['cfl'])}")
    if args.adv_flux == "lf":
        WORKLOAD.update(adv_flux=1, name=WORKLOAD["name"] + "_lf")
    if args.visc_flux == "sipg":
        WORKLOAD.update(visc_flux=1, name=WORKLOAD["name"] + "_sipg")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.impl == "reference":
        if rank == 0:
            r = run_oracle(max(1, args.steps))
            v = r["dof"] * len(r["seconds"]) / sum(r["seconds"])
            print(json.dumps({
                "impl": "reference", "metric": METRIC, "value": v, "unit": "DOF/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(r["seconds"]) / len(r["seconds"]),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded Taylor-Green state, 1e-3 perturbation)",
                "config": {"workload": WORKLOAD["name"], "arm": "oracle"},
                "cpu_baseline": {"value": v, "unit": "DOF/s", "cores": cpu_threads(), "kind": "oracle",
                                 "sample": r["sample"]},
                "e2e": {"value": v, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "gmres_iters": r["iters"], "rel_residual": r["rel_residual"]}))
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    runner = {"batched": run_batched, "mixedmesh": run_mixed_mesh, "timesteps": run_timesteps, "march": run_march,
              "peaks": run_peaks}.get(args.arm, run_ours)
    line = runner(args, world, rank, local)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and args.arm not in ("batched", "mixedmesh", "timesteps", "march", "peaks"):
            r = run_oracle(1)
            v = r["dof"] / r["seconds"][0]
            line["cpu_baseline"] = {"value": v, "unit": "DOF/s", "cores": cpu_threads(), "kind": "oracle",
                                    "sample": r["sample"], "gmres_iters": r["iters"][0]}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
