#!/usr/bin/env python3
"""Benchmark of the matrix-free high-order multigrid solver (one JSON line on rank 0).

Workload (one "step"): a full MG-preconditioned CG solve (Algorithm 1) to a 1e-8 relative
residual of the 3D variable-coefficient problem on a 16^3 hex mesh of the unit cube warped
by x_i += 0.1 prod_j sin(pi x_j), Q_4 (65^3 = 274,625 DOF incl. boundary nodes),
mu = 1 + 1e3 sum_i cos^2(2 pi x_i), seeded f ~ U(-1,1) at the nodes, V(3,3) cycles with
Chebyshev-Jacobi smoothing, FP64 throughout. The hierarchy (geometry, diagonal, Chebyshev
bounds, coarsest inverse) is built once before timing and reported as setup_ms.

value = DOF solved per second (N / solve time), whole job over all ranks (replicas).
The operator apply itself is timed separately for the roofline object.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--hier p|h] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GDOF/s of order-p operator apply; solve time to 1e-8; serve p50/p99 latency"
WORKLOAD = "3D warped var-coef Q4 16^3 (65^3=274,625 DOF), mu=1+1e3*sum cos^2(2 pi x_i), PCG + V(3,3) Chebyshev(3) to 1e-8, FP64"
# FP64 peak of one GB300: 152 SMs x 2.07 GHz x 4 FP64 flops/clock/SM (2 FMA lanes) = 1.259 TFLOP/s
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one k_apply64<3,n> launch on this workload,
# from the ncu capture summarized in profiles/apply64_fp64_q4_16cube.md (n = p + 1)
APPLY_TRAFFIC = {5: 28.744704e6}


def workload(hier):
    import synth
    return synth.warped_var3d(16, 4, hier=hier)


def oracle_sample_problem(hier):
    import synth
    return synth.warped_var3d(8, 4, hier=hier)


# ------------------------------------------------------------------ oracle arm (CPU)
def run_reference(args):
    """Time the FP64 CPU oracle (assembled sparse operators) on a bounded sample of the
    same workload: 8^3 elements instead of 16^3, same order, coefficient, warp, cycle."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    import synth
    from oracle import multigrid
    prob = oracle_sample_problem(args.hier)
    t0 = time.perf_counter()
    H = multigrid.Hierarchy(prob)
    d = H.fine.disc
    b = d.rhs(synth.nodal_field(synth.SEED_WARPED_VAR3D, d.N))
    setup_s = time.perf_counter() - t0
    times, its = [], []
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        _, it, hist, ok = H.solve_pcg(b)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            times.append(dt)
            its.append(it)
    t_step = statistics.mean(times)
    value = d.N / t_step / 1e9
    threads = int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "hier": args.hier},
        "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": threads, "kind": "oracle",
                         "sample": f"oracle PCG solve of the same warped var-coef Q4 problem on 8^3 elements "
                                   f"({d.N} DOF) instead of 16^3; setup {setup_s:.1f}s excluded; "
                                   f"{its[0]} iterations"},
        "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(hier):
    """Oracle timed in a child process on the host (single-threaded BLAS), one step."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--hier", hier],
                       capture_output=True, text=True, env=env, timeout=600)
    for ln in r.stdout.splitlines()[::-1]:
        if ln.startswith("{"):
            return json.loads(ln)["cpu_baseline"]
    return {"value": None, "unit": "GDOF/s", "cores": 1, "kind": "oracle", "sample": "failed: " + r.stderr[-300:]}


def solve_roofline_ms(P, iters, hbm_gbs, fp64_tflops, nu=(3, 3)):
    """Roofline time of one PCG + V-cycle solve (Sec. 4.2 cost model made explicit): every FP64
    apply at max(flops / FP64 peak, bytes / HBM) -- for orders 1-2 the smaller of the sum-
    factorized and the dense-element-matrix roofs -- plus the smoother updates (8 vectors per
    step), residual copies, transfers and PCG vector work at HBM speed, and the dense
    coarsest GEMV. PCG with `iters` iterations runs `iters` V-cycles and `iters` extra
    finest-level applies."""
    L = P.nlevels()
    v = (nu[0] - 1) + 1 + nu[1]
    t = 0.0
    for k in range(L):
        E3, p, N = P.level_info(k)
        dim = 3 if E3[2] > 1 or P.desc.dim == 3 else 2
        n = p + 1
        E = E3[0] * E3[1] * E3[2]
        flops = E * ((24 * n ** 4 + 15 * n ** 3) if dim == 3 else (16 * n ** 3 + 6 * n ** 2))
        nc = 6 if dim == 3 else 3
        byts = E * n ** dim * nc * 8 + 16 * N
        t_apply = max(flops / (fp64_tflops * 1e12), byts / (hbm_gbs * 1e9))
        if n <= 3:  # low orders may run from stored element matrices: the cheaper roof of the two
            d_flops, d_byts = E * 2 * n ** (2 * dim), E * 8 * n ** (2 * dim) + 16 * N
            t_apply = min(t_apply, max(d_flops / (fp64_tflops * 1e12), d_byts / (hbm_gbs * 1e9)))
        if k == L - 1:                                   # dense coarsest: one GEMV per V-cycle
            nI = 1
            for a in range(dim):
                nI *= max(0, E3[a] * p - 1)
            t += iters * (nI * nI * 8) / (hbm_gbs * 1e9)
            continue
        applies = iters * v + (iters if k == 0 else 0)
        vec = iters * (nu[0] + nu[1]) * 8 * 8 * N + iters * 6 * 8 * N   # smoother updates, copies, transfers
        if k == 0:
            vec += iters * 13 * 8 * N                     # PCG: update, dots, direction
        t += applies * t_apply + vec / (hbm_gbs * 1e9)
    return t * 1e3


# ------------------------------------------------------------------ multi-rank aggregation
def aggregate_ranks(t_step_ms, dof_per_rank, world, dist=None, device=None):
    """Replicas: every rank solves its own copy; the job's time per step is the slowest rank's
    and its throughput counts every rank's DOF: value = world * N / max_t (GDOF/s)."""
    import torch
    t = torch.tensor([float(t_step_ms)], dtype=torch.float64, device=device)
    if world > 1 and dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    return t_max, world * dof_per_rank / (t_max * 1e-3) / 1e9


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        if not self.out:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.out.strip().splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1402_5938_gb300 import Problem, launch_count

    prob = workload(args.hier)
    if args.host_loop:  # same kernels launched one by one (for launch lists; graph nodes are not listed)
        prob = dict(prob, solve_graph=0)
    t0 = time.perf_counter()
    P = Problem(prob)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    N = P.ndof(0)
    f_host = torch.from_numpy(synth.nodal_field(synth.SEED_WARPED_VAR3D, N)).pin_memory()
    f = f_host.to(dev)
    b = torch.zeros(N, dtype=torch.float64, device=dev)
    u = torch.zeros_like(b)
    P.rhs(f, b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    its = []
    for _ in range(args.warmup):
        st, it, hist = P.solve("pcg", b, u, rtol=1e-8, maxit=500)
        its.append(it)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    a0 = P.fine_applies()
    barrier()
    l0 = launch_count()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()                                   # L2 flush between timed solves
            ev[k][0].record(stream)
            st, it, hist = P.solve("pcg", b, u, rtol=1e-8, maxit=500)
            ev[k][1].record(stream)
            its.append(it)
        barrier()
    launches = launch_count() - l0
    applies = (P.fine_applies() - a0) / args.steps
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    t_step, value = aggregate_ranks(sum(step_ms) / len(step_ms), N, world, dist, dev)
    rel_res = float(hist[-1] / hist[0])

    # ---- end to end through the public API: pinned host f -> rhs -> solve -> host u
    u_host = torch.empty(N, dtype=torch.float64).pin_memory()
    e2e_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    barrier()
    e2e_ev[0].record(stream)
    for k in range(args.steps):
        f.copy_(f_host, non_blocking=True)
        P.rhs(f, b)
        P.solve("pcg", b, u, rtol=1e-8, maxit=500)
        u_host.copy_(u, non_blocking=True)
    e2e_ev[1].record(stream)
    barrier()
    _, e2e_value = aggregate_ranks(e2e_ev[0].elapsed_time(e2e_ev[1]) / args.steps, N, world, dist, dev)

    # ---- the same problem with the mixed-precision V-cycles inside FP64 PCG (context; the
    # headline value above is plain FP64): median of 5 L2-flushed solves, true FP64 residual
    mixed = {}
    for prec in (() if args.host_loop else ("fp32", "fp16", "bf16")):  # not in launch-list runs
        Pm = Problem(dict(prob, smooth_prec=prec))
        um = torch.zeros_like(b)
        for _ in range(2):
            Pm.solve("pcg", b, um, rtol=1e-8, maxit=500)
        ts = []
        for _ in range(5):
            flush.zero_()
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            stm, itm, _ = Pm.solve("pcg", b, um, rtol=1e-8, maxit=500)
            m1.record(stream)
            torch.cuda.synchronize()
            ts.append(m0.elapsed_time(m1))
        rm = torch.zeros_like(b)
        P.apply(0, um, rm)
        t_m = statistics.median(ts)
        mixed[prec] = {"solve_ms": t_m, "iterations": itm, "status": stm,
                       "fp64_rel_residual": float(torch.linalg.norm(b - rm) / torch.linalg.norm(b)),
                       "speedup_vs_fp64": t_step / t_m}
        Pm.close()

    # ---- the same problem with the other hierarchy of the configuration (h-multigrid on three
    # meshes vs p-multigrid), FP64, median of 5 L2-flushed solves (context for the headline)
    other = {}
    if not args.host_loop:
        oh = "h" if args.hier == "p" else "p"
        Po = Problem(dict(workload(oh)))
        uo = torch.zeros_like(b)
        for _ in range(2):
            Po.solve("pcg", b, uo, rtol=1e-8, maxit=500)
        ts = []
        for _ in range(5):
            flush.zero_()
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            sto, ito, _ = Po.solve("pcg", b, uo, rtol=1e-8, maxit=500)
            m1.record(stream)
            torch.cuda.synchronize()
            ts.append(m0.elapsed_time(m1))
        other = {"hier": oh, "solve_ms": statistics.median(ts), "iterations": ito, "status": sto,
                 "levels": Po.nlevels()}
        Po.close()

    # ---- the dominant kernel: the FP64 order-p apply on the finest level, timed alone
    x = torch.from_numpy(synth.uniform_pm1(7, N)).to(dev)
    y = torch.zeros_like(x)
    for _ in range(3):
        P.apply(0, x, y)
    reps = 50
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ea.record(stream)
    for _ in range(reps):
        flush.zero_()
        P.apply(0, x, y)
    eb.record(stream)
    barrier()
    ef, eg = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ef.record(stream)
    for _ in range(reps):
        flush.zero_()
    eg.record(stream)
    torch.cuda.synchronize()
    apply_ms = (ea.elapsed_time(eb) - ef.elapsed_time(eg)) / reps
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    roof_ms = solve_roofline_ms(P, its[-1], hbm, FP64_PEAK_TFLOPS)
    (E3, p, _) = P.level_info(0)
    n = p + 1
    E = E3[0] * E3[1] * E3[2]
    flops = E * (24 * n ** 4 + 15 * n ** 3)
    achieved_tf = flops / (apply_ms * 1e-3) / 1e12

    if rank == 0:
        cpu = cpu_baseline(args.hier)
        line = {
            "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "hier": args.hier, "global_batch": world, "dof": N,
                       "parallelism": f"replicas{world}", "l2": "flushed (256 MB write) between timed solves",
                       "solve_loop": "host" if args.host_loop else "graph"},
            "solve_ms": t_step, "setup_ms": setup_ms, "iterations": its[-1], "final_rel_residual": rel_res,
            "mixed_precision": mixed, "other_hierarchy": other,
            "fine_applies_per_solve": applies,
            # per PCG iteration: A p, then a V(3,3) whose pre-smoother starts from zero (2 applies),
            # the restricted residual (1) and the post-smoother (3)
            "fine_applies_model": 7 * its[-1], "apply_gdofs": N / (apply_ms * 1e-3) / 1e9,
            "apply_ms": apply_ms,
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved_tf / FP64_PEAK_TFLOPS, "traffic": APPLY_TRAFFIC.get(n),
                         "kernel": f"k_apply64<3,{n}>",
                         "note": "FP64 pipe; peak = 152 SM x 2.07 GHz x 4 flop/clk (nominal); "
                                 "algorithmic flops 24n^4+15n^3 per element"},
            "solve_roofline": {"roofline_ms": roof_ms, "measured_ms": t_step, "frac": roof_ms / t_step,
                               "model": "every apply at max(flops/FP64 peak, bytes/HBM) + vector passes and "
                                        "coarsest GEMV at HBM (HBM peak from MEASURED_PEAKS.json)"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GDOF/s", "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    P.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_sweep(args):
    """Order sweep at ~2M DOF (129^3 nodes; (64^3,2), (32^3,4), (16^3,8), (8^3,16)), same warp and
    coefficient: per order the FP64 apply time and the V-cycle operator's time in FP32, FP16 and
    BF16 (tensor cores, orders <= 7), and FP64 vs mixed-precision PCG + p-MG time to 1e-8,
    iterations, the mixed solution's FP64 residual and relative difference from the FP64 one.
    One JSON line per order (not the benchmark line)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1402_5938_gb300 import Problem
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = fn()
            b_.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b_))
        return statistics.median(ts), out

    hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    for E, p in [(64, 2), (32, 4), (16, 8), (8, 16)]:
        prob = synth.warped_var3d(E, p, hier="p")
        P64 = Problem(prob)
        N = P64.ndof(0)
        f = torch.from_numpy(synth.nodal_field(synth.SEED_PSWEEP3D, N)).to(dev)
        b = torch.zeros(N, dtype=torch.float64, device=dev)
        P64.rhs(f, b)
        y = torch.zeros_like(b)
        t64, _ = timed(lambda: P64.apply(0, b, y), 10)
        u64 = torch.zeros_like(b)
        s64, (_, it64, h64) = timed(lambda: P64.solve("pcg", b, u64, rtol=1e-8, maxit=500), 3)
        n = p + 1
        flops = E ** 3 * (24 * n ** 4 + 15 * n ** 3)
        v64, _ = P64.level_variants(0)
        line = {"sweep": f"{E}^3 Q{p}", "dof": N, "apply_fp64_ms": t64, "apply_fp64_variant": v64,
                "apply_fp64_tflops_algorithmic": flops / t64 / 1e9,
                "pcg_fp64_ms": s64, "pcg_fp64_iters": it64, "setup_bytes_fp64": P64.device_bytes()}
        if v64 == 4:
            # stored dense element matrices: 2 n^6 flops and 8 n^6 bytes per element executed
            # (fewer flops than the sum-factorized count above), so the roofline is its own
            ex_flops, ex_bytes = E ** 3 * 2 * n ** 6, E ** 3 * 8 * n ** 6 + 16 * N
            line.update({"apply_fp64_kernel": "dense element matrices",
                         "apply_fp64_frac_of_fp64_peak": ex_flops / t64 / 1e9 / FP64_PEAK_TFLOPS,
                         "apply_fp64_frac_of_hbm": ex_bytes / t64 / 1e6 / hbm_peak})
        else:
            line.update({"apply_fp64_kernel": "sum factorization",
                         "apply_fp64_frac_of_fp64_peak": flops / t64 / 1e9 / FP64_PEAK_TFLOPS})
        # V-cycle precisions: FP32, and FP16 / BF16 tensor-core applies (orders <= 7) with flexible PCG
        for prec, gbytes in (("fp32", 4), ("fp16", 2), ("bf16", 2)):
            Pm = Problem(dict(prob, smooth_prec=prec))
            x32, y32 = torch.zeros(N, dtype=torch.float32, device=dev), torch.zeros(N, dtype=torch.float32, device=dev)
            x32.copy_(b)
            tm, _ = timed(lambda: Pm.apply_f32(0, x32, y32), 10)
            um = torch.zeros_like(b)
            sm, (stm, itm, hm) = timed(lambda: Pm.solve("pcg", b, um, rtol=1e-8, maxit=500), 3)
            P64.apply(0, um, y)
            res = float(torch.linalg.norm(b - y) / torch.linalg.norm(b))
            diff = float(torch.linalg.norm(um - u64) / torch.linalg.norm(u64))
            fine_bytes = gbytes if (prec == "fp32" or p <= 7) else 4
            line.update({
                f"apply_{prec}_ms": tm, f"apply_{prec}_gdofs": N / tm / 1e6,
                f"apply_{prec}_hbm_gbs": (E ** 3 * 6 * fine_bytes * n ** 3 + 8 * N) / tm / 1e6,
                f"pcg_{prec}_ms": sm, f"pcg_{prec}_iters": itm, f"pcg_{prec}_status": stm,
                f"{prec}_speedup_vs_fp64": s64 / sm, f"{prec}_final_rel_residual_fp64": res,
                f"{prec}_vs_fp64_solution_rel_diff": diff, f"setup_bytes_{prec}": Pm.device_bytes()})
            Pm.close()
        print(json.dumps(line), flush=True)
        P64.close()
    return 0


def run_batched(args):
    """Batched workload: 512 independent 3D solves (E in 2..12, p in {2,4,6,8}, contrast 10^k,
    k in 0..4) with an FP32 V-cycle inside FP64 PCG, all through one hmg_solve_batched call, against
    the same 512 problems solved one at a time with the plain FP64 solver. One JSON line."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1402_5938_gb300 import Problem, solve_batched
    dev = torch.device("cuda", 0)
    n = args.batch
    t0 = time.perf_counter()
    mixed, fp64, bs, dofs = [], [], [], []
    for i in range(n):
        prob, seed = synth.batched_problem(i)
        Pm = Problem(prob)
        P6 = Problem(dict(prob, smooth_prec="fp64"))
        N = Pm.ndof(0)
        b = torch.zeros(N, dtype=torch.float64, device=dev)
        Pm.rhs(torch.from_numpy(synth.nodal_field(seed, N)).to(dev), b)
        mixed.append(Pm)
        fp64.append(P6)
        bs.append(b)
        dofs.append(N)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    us = [torch.zeros_like(b) for b in bs]
    solve_batched(mixed, "pcg", bs, us, rtol=1e-8, maxit=500)          # builds the graphs
    reps, tb = 3, []
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        sts, its, _ = solve_batched(mixed, "pcg", bs, us, rtol=1e-8, maxit=500)
        tb.append(time.perf_counter() - t)
    u6 = [torch.zeros_like(b) for b in bs]
    for P, b, u in zip(fp64, bs, u6):                                   # build graphs
        P.solve("pcg", b, u, rtol=1e-8, maxit=500)
    torch.cuda.synchronize()
    t = time.perf_counter()
    its6 = []
    for P, b, u in zip(fp64, bs, u6):
        st, it, _ = P.solve("pcg", b, u, rtol=1e-8, maxit=500)
        its6.append(it)
    t_seq = time.perf_counter() - t
    diff = max(float(torch.linalg.norm(a - c) / torch.linalg.norm(c)) for a, c in zip(us, u6))
    r = torch.zeros_like(bs[0])
    worst = 0.0
    for P, b, u in zip(fp64, bs, us):
        rr = torch.zeros_like(b)
        P.apply(0, u, rr)
        worst = max(worst, float(torch.linalg.norm(b - rr) / torch.linalg.norm(b)))
    tbm = statistics.median(tb)
    print(json.dumps({
        "batched": f"{n} solves", "total_dof": sum(dofs), "setup_s_both_sets": setup_s,
        "batched_mixed_s": tbm, "batched_solves_per_s": n / tbm, "batched_gdof_per_s": sum(dofs) / tbm / 1e9,
        "fp64_one_at_a_time_s": t_seq, "fp64_solves_per_s": n / t_seq, "speedup_vs_fp64_sequential": t_seq / tbm,
        "all_converged": all(s_ == 0 for s_ in sts), "iters_mixed_mean": statistics.mean(its),
        "iters_fp64_mean": statistics.mean(its6), "max_rel_diff_mixed_vs_fp64": diff,
        "worst_fp64_residual_of_mixed": worst}), flush=True)
    for P in mixed + fp64:
        P.close()
    return 0


def run_serve(args):
    """Serving workload: Poisson arrivals (2,000/s mean) of 2D/3D solves, DOF log-uniform in
    [1e3, 2e6], p uniform in 1..16, through the continuous-batching server (FP32 V-cycle in FP64
    PCG); p50/p99 latency (submit to result on the host) and solves/s at the specified rate and
    at half the measured saturated rate, against the plain FP64 path one request at a time
    (single-server queue on the same arrivals). One JSON line."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1402_5938_gb300 import Problem, Server, desc_ndof
    dev = torch.device("cuda", 0)
    R = args.requests
    reqs = [synth.serving_request(i) for i in range(R)]
    fs = [synth.nodal_field(seed, desc_ndof(prob)) for prob, seed, _ in reqs]
    gaps = np.array([g for _, _, g in reqs])

    def serve(scale, slots):
        srv = Server(0, 160 << 30, slots)
        arr = np.cumsum(gaps * scale)
        t0 = time.perf_counter()
        tickets = []
        for (prob, _, _), f, a in zip(reqs, fs, arr):
            dt = t0 + a - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(prob, f, rtol=1e-8, mode="pcg", maxit=500))
        lat, ok, done_at, failed = [], 0, [], []
        for i, ((t, n), a) in enumerate(zip(tickets, arr)):
            st, u, it, res, l = srv.wait(t, n)
            ok += int(st == 0)
            if st != 0:
                p = reqs[i][0]
                failed.append({"i": i, "status": st, "iters": it, "dim": p["dim"], "nelem": p["nelem"][0],
                               "order": p["order"], "res": res})
            lat.append(l)
            done_at.append(a + l)
        span = max(done_at)
        srv.close()
        return dict(p50_ms=1e3 * float(np.percentile(lat, 50)), p99_ms=1e3 * float(np.percentile(lat, 99)),
                    solves_per_s=R / span, ok=ok, offered_per_s=R / arr[-1], failed=failed)

    hot = serve(1.0, args.slots)
    cool = serve(max(1.0, (R / gaps.sum()) / (0.5 * hot["solves_per_s"])), args.slots)
    # plain FP64 path, one request at a time: service times, then a single-server queue
    service = []
    for (prob, _, _), f in zip(reqs, fs):
        torch.cuda.synchronize()
        t = time.perf_counter()
        P = Problem(dict(prob, smooth_prec="fp64"))
        N = P.ndof(0)
        b = torch.zeros(N, dtype=torch.float64, device=dev)
        P.rhs(torch.from_numpy(f).to(dev), b)
        u = torch.zeros_like(b)
        P.solve("pcg", b, u, rtol=1e-8, maxit=500)
        u.cpu()
        P.close()
        service.append(time.perf_counter() - t)
    arr = np.cumsum(gaps)
    fin, lat = 0.0, []
    for a, sv in zip(arr, service):
        start = max(a, fin)
        fin = start + sv
        lat.append(fin - a)
    print(json.dumps({
        "serve": f"{R} requests, Poisson 2000/s, {args.slots} slots", "at_2000_per_s": hot,
        "below_saturation": cool,
        "fp64_one_at_a_time": {"p50_ms": 1e3 * float(np.percentile(lat, 50)),
                               "p99_ms": 1e3 * float(np.percentile(lat, 99)), "solves_per_s": R / fin,
                               "mean_service_ms": 1e3 * float(np.mean(service))}}), flush=True)
    return 0


def paper_table_counts(tab, p, key):
    """Iteration count of one cell of the paper's Table 1 (2d-const) / Table 4 (3d-const) from the
    GPU solver: unit square/cube, mu = 1, three meshes, (3,3) smoothing, seeded U(-1,1) load."""
    import torch

    import synth
    from paper_1402_5938_gb300 import Problem
    mode, smoother, hier = key.split()
    dim, nelem = (2, 32) if tab == "table1_2d_const" else (3, 8)
    prob = synth.problem(dim, nelem, p, hier=hier, smoother=smoother, nu_pre=3, nu_post=3)
    P = Problem(prob)
    N = P.ndof(0)
    b = torch.zeros(N, dtype=torch.float64, device="cuda")
    P.rhs(torch.from_numpy(synth.nodal_field(7, N)).cuda(), b)
    u = torch.zeros_like(b)
    st, it, _ = P.solve(mode.lower(), b, u, rtol=1e-8, maxit=500)
    P.close()
    return it if st == 0 else None


def run_paper_tables(args):
    """Tables 1 and 4 of the paper (point-smoother columns) and Table 7's 2d-const point / l1-Jacobi
    rows recomputed on the GPU; prints markdown tables (GPU count / paper count) and one JSON
    summary line."""
    import __graft_entry__
    __graft_entry__.build()
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_tables.json")))
    keys = ["MG jacobi h", "MG jacobi p", "MG cheb h", "MG cheb p",
            "PCG jacobi h", "PCG jacobi p", "PCG cheb h", "PCG cheb p"]
    worst, cells = 0, 0
    for tab in ("table1_2d_const", "table4_3d_const"):
        print(f"\n{tab} (GPU / paper)\n")
        print("| p | " + " | ".join(keys) + " |")
        print("|---" * (len(keys) + 1) + "|")
        for p in (1, 2, 3, 4, 5, 6, 7, 8, 16):
            row = []
            for key in keys:
                ref = gold[tab][key].get(str(p))
                # the 3D order-16 h-hierarchy ends on 31^3 = 29,791 unknowns: beyond the dense
                # exact coarsest solve (20,000); the 2D one (127^2 = 16,129) runs
                if ref is None or (p == 16 and key.endswith(" h") and tab == "table4_3d_const"):
                    row.append("" if ref is None else f"n/a / {ref}")
                    continue
                it = paper_table_counts(tab, p, key)
                row.append(f"{it} / {ref}")
                worst = max(worst, abs((it if it is not None else 10 ** 6) - ref))
                cells += 1
            print(f"| {p} | " + " | ".join(row) + " |", flush=True)
    # Table 7, 2d-const rows: point, element-block and l1-Jacobi, h-multigrid on 32^2, MG and PCG;
    # beside the counts, the GPU time to solution of each (graph solve, median of 3)
    import torch

    import synth
    from paper_1402_5938_gb300 import Problem
    t7 = gold["table7_l1_2d_const"]
    t7b = gold["table7_block_2d_const"]
    print("\ntable7_2d_const (GPU / paper; GPU ms to 1e-8)\n")
    print("| p | pt MG | pt PCG | blk MG | blk PCG | l1 MG | l1 PCG | PCG ms pt / blk / l1 | setup ms pt / blk / l1 |")
    print("|---|---|---|---|---|---|---|---|---|")
    ratios, bratios, times = {}, {}, {}
    for p in (8, 16):
        got, ms, setup = {}, {}, {}
        for sm, col in (("jacobi", "pt"), ("blockjacobi", "blk"), ("l1jacobi", "l1")):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            P = Problem(synth.problem(2, 32, p, hier="h", n_hlevels=3, smoother=sm, nu_pre=3, nu_post=3))
            torch.cuda.synchronize()
            setup[col] = (time.perf_counter() - t0) * 1e3
            N = P.ndof(0)
            b = torch.zeros(N, dtype=torch.float64, device="cuda")
            P.rhs(torch.from_numpy(synth.nodal_field(7, N)).cuda(), b)
            for mode in ("MG", "PCG"):
                u = torch.zeros_like(b)
                st, it, _ = P.solve(mode.lower(), b, u, rtol=1e-8, maxit=1000)
                got[(col, mode)] = it if st == 0 else None
            tt = []
            for _ in range(3):
                u = torch.zeros_like(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                P.solve("pcg", b, u, rtol=1e-8, maxit=1000)
                torch.cuda.synchronize()
                tt.append((time.perf_counter() - t0) * 1e3)
            ms[col] = sorted(tt)[1]
            P.close()
        gold_of = lambda c_, m: (t7b if c_ == "blk" else t7)[c_][m][str(p)]
        print(f"| {p} | " + " | ".join(f"{got[(c_, m)]} / {gold_of(c_, m)}"
                                        for c_ in ("pt", "blk", "l1") for m in ("MG", "PCG")) +
              f" | {ms['pt']:.2f} / {ms['blk']:.2f} / {ms['l1']:.2f} | {setup['pt']:.0f} / {setup['blk']:.0f} / {setup['l1']:.0f} |",
              flush=True)
        ratios[p] = {m: [got[("l1", m)] / got[("pt", m)], t7["l1"][m][str(p)] / t7["pt"][m][str(p)]] for m in ("MG", "PCG")}
        bratios[p] = {m: [got[("blk", m)] / got[("pt", m)], t7b["blk"][m][str(p)] / t7b["pt"][m][str(p)]]
                      for m in ("MG", "PCG")}
        times[p] = {"pcg_ms": ms, "setup_ms": setup}
    # Table 1's last column: CG preconditioned by the low-order operator (Q1 on the order-p nodes),
    # inverted by its own multigrid-preconditioned CG to 1e-12 (the paper factors it)
    tl = gold["table1_low_order_2d_const"]["PCG"]
    print("\ntable1_low_order_2d_const (GPU / paper; inner CG iterations in total; GPU ms)\n")
    print("| p | low-order PCG | inner iterations | ms |")
    print("|---|---|---|---|")
    low_counts = {}
    for p in (2, 3, 4, 5, 6, 7, 8, 16):
        prob = synth.problem(2, 32, p, hier="p", n_hlevels=1)   # only its finest operator is used
        P = Problem(prob)
        N = P.ndof(0)
        xyz = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
        P.node_coords(0, xyz)
        lo = Problem(synth.low_order_problem(prob, xyz.cpu().numpy().reshape(2, N)))
        b = torch.zeros(N, dtype=torch.float64, device="cuda")
        P.rhs(torch.from_numpy(synth.nodal_field(7, N)).cuda(), b)
        u = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it, inner, _ = P.solve_low_order(lo, b, u, rtol=1e-8)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        low_counts[p] = it if st == 0 else None
        if st == 0:
            worst = max(worst, abs(it - tl[str(p)]))
            cells += 1
        print(f"| {p} | {low_counts[p]} / {tl[str(p)]} | {inner} | {ms:.1f} |", flush=True)
        lo.close()
        P.close()
    print(json.dumps({"paper_tables": "Tables 1, 4 and 7", "cells": cells, "max_abs_diff": worst,
                      "table1_low_order_gpu": low_counts,
                      "table7_l1_over_point_ratios_gpu_vs_paper": ratios,
                      "table7_block_over_point_ratios_gpu_vs_paper": bratios,
                      "table7_times_gpu": times}), flush=True)
    return 0


def run_block_jacobi(args):
    """Element-block Jacobi on the GPU: the zero-guess smoothing step (block inverses on element
    interiors + point step on shared nodes) against the HBM roofline, and PCG time to 1e-8 with
    block, point Jacobi and Chebyshev smoothing on the same problems. One JSON line per problem."""
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1402_5938_gb300 import Problem
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    cases = [("2d-const 128^2 Q8, h-MG 5 levels", synth.problem(2, 128, 8, hier="h", n_hlevels=5)),
             ("2d-const 32^2 Q16, h-MG 3 levels", synth.problem(2, 32, 16, hier="h", n_hlevels=3)),
             ("3d-var warped 16^3 Q4, p-MG", synth.warped_var3d(16, 4, hier="p")),
             ("3d-var warped 8^3 Q8, p-MG", synth.warped_var3d(8, 8, hier="p"))]
    for ci, (name, base) in enumerate(cases):
        if args.block_case >= 0 and ci != args.block_case:
            continue
        out = {"block_jacobi": name}
        for sm in ("blockjacobi", "jacobi", "cheb"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            P = Problem(dict(base, smoother=sm))
            torch.cuda.synchronize()
            setup_ms = (time.perf_counter() - t0) * 1e3
            N = P.ndof(0)
            b = torch.zeros(N, dtype=torch.float64, device="cuda")
            P.rhs(torch.from_numpy(synth.nodal_field(3, N)).cuda(), b)
            u = torch.zeros_like(b)
            st, it, _ = P.solve("pcg", b, u, rtol=1e-8, maxit=1000)
            tt = []
            for _ in range(5):
                u.zero_()
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                P.solve("pcg", b, u, rtol=1e-8, maxit=1000)
                torch.cuda.synchronize()
                tt.append((time.perf_counter() - t0) * 1e3)
            out[sm] = {"pcg_iterations": it, "status": st, "pcg_ms": statistics.median(tt), "setup_ms": setup_ms}
            if sm == "blockjacobi":
                # one zero-guess step on the finest level: x = omega (D_s^-1 b + blockdiag(K_II^-1) b)
                d, E, p = base["dim"], 1, base["order"]
                for e in base["nelem"]:
                    E *= e
                mi = (p - 1) ** d
                # block inverses (packed, column pairs), interior gather / x read-modify-write, point step
                byts = E * ((mi + 1) // 2) * 2 * mi * 8 + E * mi * 24 + N * 24
                flops = 2 * E * mi * mi + 2 * N
                # the GEMV does 2 flops per 8-byte entry, above GB300's FP64 ridge (~0.19 flop/B):
                # its roof is the FP64 pipe unless the bytes take longer
                t_hbm = byts / (hbm * 1e9)
                t_fp64 = flops / (FP64_PEAK_TFLOPS * 1e12)
                x = torch.zeros_like(b)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ts = []
                for _ in range(10):
                    flush.sum()   # evict by reading: no dirty lines left to write back in the timed region
                    torch.cuda.synchronize()
                    ev[0].record()
                    P.smooth(0, b, x, 1, zero_guess=True)
                    ev[1].record()
                    torch.cuda.synchronize()
                    ts.append(ev[0].elapsed_time(ev[1]))
                step_ms = statistics.median(ts[3:])
                out["block_step"] = {"ms": step_ms, "bytes": byts, "flops": flops,
                                     "bound": "fp64" if t_fp64 >= t_hbm else "hbm",
                                     "roof_ms": max(t_hbm, t_fp64) * 1e3,
                                     "frac": max(t_hbm, t_fp64) / (step_ms * 1e-3),
                                     "achieved_gbs": byts / (step_ms * 1e-3) / 1e9, "peak_gbs": hbm,
                                     "achieved_tflops": flops / (step_ms * 1e-3) / 1e12,
                                     "peak_tflops": FP64_PEAK_TFLOPS,
                                     "kernels": "k_jacobi_first + k_block_smooth (zero guess, 1 step)"}
            P.close()
        print(json.dumps(out), flush=True)
    return 0


def run_spectral(args):
    """The paper's smoother / two-grid spectral study (Figs. 2-3) on the GPU: for 2d-const and
    2d-var at p = 1, 4, 16 (961 interior unknowns each), the interior matrix A is assembled by
    applying the GPU operator to unit vectors and its eigenvectors v_i taken with numpy; then the
    error propagators of six smoothing steps (hmg_smooth) and of one two-grid cycle (hmg_vcycle
    on two h-levels, exact coarse solve) are applied to every v_i on the GPU. Reported per
    smoother: ||S V_upper||_2 (damping of the upper half of the spectrum), the number of singular
    values of S below 0.1, the two-grid spectral radius rho(T), and the figures' own data -- the
    largest coefficient of T sum_i v_i and how many exceed 1 -- with each v_i's largest entry made
    positive (that data depends on such a choice; the other three do not)."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_1402_5938_gb300 import Problem
    smoothers = ("jacobi", "cheb", "l1jacobi", "blockjacobi")
    summary = {}
    print("\n| problem | p | smoother | \\|\\|S V_upper\\|\\| | #sigma(S) < 0.1 | rho(T) two-grid | "
          "max \\|c\\| of T sum v_i | #\\|c\\| > 1 |")
    print("|---|---|---|---|---|---|---|---|")
    for kind in ("2d-const", "2d-var"):
        for p in (1, 4, 16):
            for sm in smoothers:
                P = Problem(synth.spectral_problem(kind, p, sm))
                N = P.ndof(0)
                n1 = round(N ** 0.5)
                interior = np.arange(N).reshape(n1, n1)[1:-1, 1:-1].ravel()
                idx = torch.from_numpy(interior).cuda()
                n = len(interior)
                A = np.empty((n, n))
                x = torch.zeros(N, dtype=torch.float64, device="cuda")
                y, z, zero = torch.zeros_like(x), torch.zeros_like(x), torch.zeros_like(x)
                for j, g in enumerate(interior):
                    x.zero_()
                    x[int(g)] = 1.0
                    P.apply(0, x, y)
                    A[:, j] = y[idx].cpu().numpy()
                lam, V = np.linalg.eigh(0.5 * (A + A.T))
                V *= np.where(V[np.abs(V).argmax(axis=0), np.arange(n)] < 0, -1.0, 1.0)[None, :]
                S, T = np.empty((n, n)), np.empty((n, n))
                for j in range(n):
                    x.zero_()
                    x[idx] = torch.from_numpy(V[:, j]).cuda()
                    P.apply(0, x, y)
                    z.zero_()
                    P.vcycle(-y, z)
                    T[:, j] = (x + z)[idx].cpu().numpy()
                    P.smooth(0, zero, x, 6)
                    S[:, j] = x[idx].cpu().numpy()
                Ms, Mt = V.T @ S, V.T @ T
                c = Mt @ np.ones(n)
                row = {"smooth_norm_upper": float(np.linalg.norm(Ms[:, n // 2:], 2)),
                       "smooth_sigma_below_0.1": int(np.sum(np.linalg.svd(Ms, compute_uv=False) < 0.1)),
                       "twogrid_rho": float(np.abs(np.linalg.eigvals(Mt)).max()),
                       "figure_max_coef": float(np.abs(c).max()), "figure_coefs_above_1": int(np.sum(np.abs(c) > 1.0))}
                summary[f"{kind} p{p} {sm}"] = row
                print(f"| {kind} | {p} | {sm} | {row['smooth_norm_upper']:.3f} | {row['smooth_sigma_below_0.1']} | "
                      f"{row['twogrid_rho']:.3f} | {row['figure_max_coef']:.3f} | {row['figure_coefs_above_1']} |",
                      flush=True)
                P.close()
    print(json.dumps({"spectral": "Figs. 2-3 setting, 961 unknowns, 6 smoothing steps / two-grid V(3,3)",
                      "cases": summary}), flush=True)
    return 0


def run_mesh_independence(args):
    """Mesh independence (the paper's Table 6 setting with this library's smoothers): PCG with an
    h-multigrid V(3,3) down to 2 x 2 elements on 2D meshes E x E, E = 4..256, orders 1..16, for
    2d-const and 2d-var and point Jacobi / Chebyshev smoothing. Prints markdown tables with the
    paper's SSOR(2,1) counts beside (context) and one JSON summary line."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1402_5938_gb300 import Problem
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_tables.json")))["table6_mesh_independence"]
    Es = gold["E"]
    spread = {}
    for kind in ("2d-const", "2d-var"):
        for smoother in ("jacobi", "cheb"):
            print(f"\n{kind}, PCG + h-MG V(3,3) {smoother} (GPU count / paper SSOR(2,1) count)\n")
            print("| p | " + " | ".join(f"E={E}" for E in Es) + " |")
            print("|---" * (len(Es) + 1) + "|")
            for p in (1, 2, 4, 8, 16):
                row, counts = [], []
                for E, ref in zip(Es, gold[kind][str(p)]):
                    P = Problem(synth.mesh_independence_problem(kind, E, p, smoother))
                    N = P.ndof(0)
                    b = torch.zeros(N, dtype=torch.float64, device="cuda")
                    P.rhs(torch.from_numpy(synth.nodal_field(11, N)).cuda(), b)
                    u = torch.zeros_like(b)
                    st, it, _ = P.solve("pcg", b, u, rtol=1e-8, maxit=300)
                    P.close()
                    counts.append(it if st == 0 else None)
                    row.append(f"{it if st == 0 else '-'} / {ref if ref is not None else '*'}")
                ok = [k for k, E in zip(counts, Es) if E >= 16 and k is not None]
                spread[f"{kind} {smoother} p{p}"] = (max(ok) - min(ok)) if ok else None
                print(f"| {p} | " + " | ".join(row) + " |", flush=True)
    print(json.dumps({"mesh_independence": "PCG + h-MG V(3,3) to 2x2 elements, E = 4..256",
                      "max_spread_E_ge_16": max(v for v in spread.values() if v is not None),
                      "spread": spread}), flush=True)
    return 0


def run_profile_apply(args):
    """Small fixed launch sequence for ncu: build the hierarchy of the warped var-coef problem
    (--mesh elements per axis, --order p, p-multigrid), then two applies on each of the three
    finest levels (FP64 hmg_apply, or hmg_apply_f32 with --prec fp32/fp16/bf16) after setup's applies."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1402_5938_gb300 import Problem
    prob = synth.warped_var3d(args.mesh, args.order, hier=args.hier)
    if args.prec != "fp64":
        prob = dict(prob, smooth_prec=args.prec)
    P = Problem(prob)
    for lev in range(min(3, P.nlevels())):
        N = P.ndof(lev)
        x = torch.from_numpy(synth.uniform_pm1(7, N)).cuda()
        y = torch.zeros_like(x)
        for _ in range(2):
            if args.prec != "fp64":
                P.apply_f32(lev, x.float(), y.float())
            else:
                P.apply(lev, x, y)
    torch.cuda.synchronize()
    P.close()
    print("profile-apply ok")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--hier", choices=["h", "p"], default="p")
    ap.add_argument("--host-loop", action="store_true",
                    help="host-driven solve loop instead of the graph (for ncu launch lists)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--profile-apply", action="store_true", help="launch sequence for ncu captures")
    ap.add_argument("--sweep", action="store_true", help="order sweep at ~2M DOF, FP64 vs mixed precision")
    ap.add_argument("--paper-tables", action="store_true", help="the paper's Tables 1 and 4 recomputed on the GPU")
    ap.add_argument("--mesh-independence", action="store_true",
                    help="Table 6 setting: iterations vs fine mesh at a fixed 2x2 coarsest grid")
    ap.add_argument("--batched", action="store_true", help="512-solve batched workload vs FP64 one at a time")
    ap.add_argument("--block-jacobi", action="store_true", help="element-block Jacobi: step roofline, solve times")
    ap.add_argument("--spectral", action="store_true", help="the paper's Figs. 2-3 smoother / two-grid spectral study")
    ap.add_argument("--block-case", type=int, default=-1, help="--block-jacobi: run only this problem (0..3)")
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--serve", action="store_true", help="Poisson-arrival serving workload")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--mesh", type=int, default=16, help="--profile-apply: elements per axis")
    ap.add_argument("--order", type=int, default=4, help="--profile-apply: polynomial order")
    ap.add_argument("--prec", choices=["fp64", "fp32", "fp16", "bf16"], default="fp64",
                    help="--profile-apply: precision")
    args = ap.parse_args()
    if args.sweep:
        return run_sweep(args)
    if args.batched:
        return run_batched(args)
    if args.paper_tables:
        return run_paper_tables(args)
    if args.mesh_independence:
        return run_mesh_independence(args)
    if args.block_jacobi:
        return run_block_jacobi(args)
    if args.spectral:
        return run_spectral(args)
    if args.serve:
        return run_serve(args)
    if args.profile_apply:
        return run_profile_apply(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
