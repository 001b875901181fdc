#!/usr/bin/env python3
"""Benchmark of the matrix-free high-order multigrid solver (one JSON line on rank 0).

Workload: the ~2M-DOF configuration of the order sweep at p = 4 -- a 32^3 hex mesh of the
unit cube warped by x_i += 0.1 prod_j sin(pi x_j), Q_4 (129^3 = 2,146,689 DOF incl. boundary
nodes), mu = 1 + 1e3 sum_i cos^2(2 pi x_i), seeded f ~ U(-1,1) at the nodes, p-multigrid
(Q4 -> Q2 -> Q1, then two mesh halvings) V(3,3) Chebyshev-Jacobi as the PCG preconditioner,
FP64 throughout. The hierarchy (geometry, diagonal, Chebyshev bounds, coarsest inverse) is
built once before timing and reported as setup_ms.

One step = one pass of the whole hot path: the finest-level operator apply y = A x timed on
its own (CUDA events), then the PCG solve to a 1e-8 relative residual (gather/scatter, sum
factorization, smoothers, transfers, coarsest solve, V-cycles inside Algorithm 1).
value = GDOF/s of the order-p operator apply (N / apply time), whole job over all ranks
(replicas); solve_ms = time to 1e-8 of the same step. e2e: the same apply through the host-
buffer call hmg_apply_host (page-locked x in, y out, copies inside the timed region), and the
solve through hmg_solve_host (nodal f in, u out). Further blocks: the same problem's FP32 /
FP16 / BF16 V-cycles inside FP64 PCG, the finest FP64 operator in double-float arithmetic (its
apply, and PCG with the FP64 / FP32 / FP16 V-cycles), the order sweep at 129^3 nodes (p = 2, 8,
16), and the 16^3 Q4 (274,625 DOF) single-solve configuration with its h- and p-hierarchies.

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
WORKLOAD = ("3D warped var-coef Q4 32^3 (129^3=2,146,689 DOF), mu=1+1e3*sum cos^2(2 pi x_i), "
            "p-MG PCG + V(3,3) Chebyshev(3) to 1e-8, FP64")
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the headline's FP64 apply kernel, by
# (kernel, elements): per launch, from the ncu capture named in "traffic_source"; None when the
# kernel has changed since that capture
APPLY_TRAFFIC = {("k_apply64<3,5,2>", 32768): 229.953024e6 + 12.929792e6}
TRAFFIC_SOURCE = "ncu capture of k_apply64<3,5,2> on the 32^3 Q4 level: dram__bytes_read.sum + dram__bytes_write.sum"
REF_ROWS_PER_STEP = 400


class L2Flush:
    """Between timed iterations: write a buffer larger than L2 (256 MB), then read a second one, so
    that L2 holds none of the timed kernel's data and no dirty lines whose write-back would land in
    the timed region."""

    def __init__(self, device):
        import torch
        self.w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
        self.r = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def zero_(self):
        self.w.zero_()
        self.r.sum()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def workload(hier, nelem=32, order=4):
    import synth
    return synth.warped_var3d(nelem, order, hier=hier)


# ------------------------------------------------------------------ oracle arm (CPU)
def run_reference(args):
    """The FP64 CPU oracle on the same workload and metric: sampled rows of the order-p operator
    apply y = A x by the oracle's weak form (Sec. 2.1, evaluated per row from the element
    geometry and dense basis tables, no assembly: the assembled operator of 129^3 nodes does not
    fit a bounded sample), REF_ROWS_PER_STEP rows per step, single-threaded."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    import numpy as np

    import synth
    from oracle import fem
    prob = workload(args.hier)
    t0 = time.perf_counter()
    d = fem.Discretization(3, prob["nelem"], prob["order"], warp_amp=prob["warp_amp"], mu_a=prob["mu_a"],
                           mu_b=prob["mu_b"], mu_k=prob["mu_k"])
    x = synth.uniform_pm1(7, d.N)
    d.node_coords_cached()
    setup_s = time.perf_counter() - t0
    rng = np.random.default_rng(12)
    times = []
    rows_per = args.ref_rows
    for k in range(args.warmup + args.steps):
        rows = d.interior[rng.choice(d.n_interior, rows_per, replace=False)]
        t = time.perf_counter()
        d.apply_rows(x, rows)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            times.append(dt)
    t_step = statistics.mean(times)
    value = rows_per / t_step / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "hier": args.hier, "dof": d.N},
        "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": 1, "nproc": os.cpu_count(), "kind": "oracle",
                         "sample": f"oracle order-4 apply (weak form per row) on {rows_per} random interior rows "
                                   f"per step of the same {d.N}-DOF problem, single thread; setup "
                                   f"{setup_s:.1f}s excluded"},
        "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(hier, steps=10):
    """The oracle arm in a child process on the host (single thread), steps x REF_ROWS_PER_STEP rows."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", str(steps), "--warmup", "1", "--hier", hier],
                       capture_output=True, text=True, env=env, timeout=900)
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
_PEAK = {}


def fp64_peak():
    """Measured FP64 FMA rate of this GPU in TFLOP/s (hmg_measure_peak), once per process."""
    if "fp64" not in _PEAK:
        from paper_1402_5938_gb300 import measure_peak
        _PEAK["fp64"] = measure_peak("fp64")
    return _PEAK["fp64"]


def flop_per_elem(dim, n):
    """Algorithmic flops of one element's sum-factorized apply (a3-a5): 24n^4 + 15n^3 in 3D."""
    return (24 * n ** 4 + 15 * n ** 3) if dim == 3 else (16 * n ** 3 + 6 * n ** 2)


def events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def timed_solves(P, b, u, flush, stream, reps, warm=2, mode="pcg"):
    """Median ms of `reps` L2-flushed solves (after `warm` untimed ones), last status and iterations."""
    import torch
    for _ in range(warm):
        P.solve(mode, b, u, rtol=1e-8, maxit=500)
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = events(2)
        e0.record(stream)
        st, it, _ = P.solve(mode, b, u, rtol=1e-8, maxit=500)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), st, it


def timed_apply(fn, flush, stream, reps):
    """Median ms of `reps` L2-flushed calls of fn (one operator apply each)."""
    import torch
    fn()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = events(2)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def mixed_block(prob, P64, b, flush, stream, t64_ms, reps=5):
    """The same problem solved with the FP32, FP16 and BF16 V-cycles inside FP64 PCG: solve time,
    iterations, the true FP64 residual of the mixed solution, and the V-cycle operator's apply."""
    import torch
    out = {}
    N = b.numel()
    for prec in ("fp32", "fp16", "bf16"):
        Pm = __import__("paper_1402_5938_gb300").Problem(dict(prob, smooth_prec=prec))
        um = torch.zeros_like(b)
        t, st, it = timed_solves(Pm, b, um, flush, stream, reps)
        rm = torch.zeros_like(b)
        P64.apply(0, um, rm)
        x32 = b.float()
        y32 = torch.zeros_like(x32)
        ta = timed_apply(lambda: Pm.apply_f32(0, x32, y32), flush, stream, 10)
        (E3, p, _) = Pm.level_info(0)
        dim = 3 if E3[2] > 1 or prob["dim"] == 3 else 2
        E = E3[0] * E3[1] * E3[2]
        # algorithmic bytes of the V-cycle operator: its geometric factors (FP32 or 16-bit) once,
        # x read and y written once in FP32
        fbytes = E * (p + 1) ** dim * (6 if dim == 3 else 3) * (4 if prec == "fp32" else 2) + 8 * N
        hbm = measured_peaks().get("hbm_gbs", 6800.0)
        out[prec] = {"solve_ms": t, "iterations": it, "status": st,
                     "fp64_rel_residual": float(torch.linalg.norm(b - rm) / torch.linalg.norm(b)),
                     "speedup_vs_fp64": t64_ms / t, "fine_apply_ms": ta, "fine_apply_gdofs": N / (ta * 1e-3) / 1e9,
                     "fine_apply_variant": Pm.level_variants(0)[1], "fine_apply_bytes": fbytes,
                     "fine_apply_frac_of_hbm": fbytes / (ta * 1e-3) / 1e9 / hbm,
                     "fine_apply_note": "hmg_apply_f32 (zeroing y + the pencil-form kernel), CUDA events, L2 flushed"}
        Pm.close()
    return out


def df64_block(prob, P64, b, flush, stream, t64_ms, apply64_ms, peak64, reps=5):
    """The finest level's FP64 operator in double-float arithmetic (fp64_arith = df64: pairs of FP32
    numbers, FP64 vectors, the FP64 factors split into float pairs): its apply against the native
    FP64 apply of the timed steps, and PCG solves with the FP64, FP32 and FP16 V-cycles (solve time,
    iterations, the true FP64 residual of the solution by the native FP64 operator)."""
    import torch
    Problem = __import__("paper_1402_5938_gb300").Problem
    N = b.numel()
    Pd = Problem(dict(prob, fp64_arith="df64"))
    yd = torch.zeros_like(b)
    ta = timed_apply(lambda: Pd.apply(0, b, yd), flush, stream, 20)
    y64 = torch.zeros_like(b)
    P64.apply(0, b, y64)
    Pd.apply(0, b, yd)
    (E3, p, _) = Pd.level_info(0)
    flops = E3[0] * E3[1] * E3[2] * flop_per_elem(3, p + 1)
    out = {"apply_ms": ta, "apply_fp64_ms": apply64_ms, "speedup_vs_fp64_apply": apply64_ms / ta,
           "apply_gdofs": N / (ta * 1e-3) / 1e9, "fp64_equivalent_tflops": flops / (ta * 1e-3) / 1e12,
           "fp64_peak_tflops": peak64, "variant": Pd.level_variants(0)[0],
           "max_rel_diff_vs_fp64": float((yd - y64).abs().max() / y64.abs().max()),
           "arith": "double-float: pairs of FP32 numbers (about 48 significant bits), FP64 vectors in and out",
           "note": "hmg_apply with CUDA events, L2 flushed; fp64_equivalent_tflops = the FP64 operator's "
                   "algorithmic flops (24n^4+15n^3 per element) / time",
           "solves": {}}
    Pd.close()
    for prec in ("fp64", "fp32", "fp16"):
        Pm = Problem(dict(prob, smooth_prec=prec, fp64_arith="df64"))
        um = torch.zeros_like(b)
        t, st, it = timed_solves(Pm, b, um, flush, stream, reps)
        r = torch.zeros_like(b)
        P64.apply(0, um, r)
        out["solves"][prec + "_v_cycle"] = {
            "solve_ms": t, "iterations": it, "status": st, "speedup_vs_fp64": t64_ms / t,
            "fp64_rel_residual": float(torch.linalg.norm(b - r) / torch.linalg.norm(b))}
        Pm.close()
    return out


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

    peak64 = fp64_peak()
    prob = workload(args.hier)
    if args.host_loop:  # same kernels launched one by one (for launch lists; graph nodes are not listed)
        prob = dict(prob, solve_graph=0)
        if args.prec != "fp64":  # the launch list of a mixed-precision solve
            prob = dict(prob, smooth_prec=args.prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P = Problem(prob)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    N = P.ndof(0)
    f_host = torch.from_numpy(synth.nodal_field(synth.SEED_PSWEEP3D, N)).pin_memory()
    f = f_host.to(dev)
    b = torch.zeros(N, dtype=torch.float64, device=dev)
    u = torch.zeros_like(b)
    P.rhs(f, b)
    x = torch.from_numpy(synth.uniform_pm1(7, N)).to(dev)
    y = torch.zeros_like(x)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    its = []
    for _ in range(args.warmup):
        P.apply(0, x, y)
        st, it, hist = P.solve("pcg", b, u, rtol=1e-8, maxit=500)
        its.append(it)
    ev = [events(3) for _ in range(args.steps)]
    a0 = P.fine_applies()
    barrier()
    l0 = launch_count()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()                                   # L2 flush between timed steps
            ev[k][0].record(stream)
            P.apply(0, x, y)                                # the order-p operator apply
            ev[k][1].record(stream)
            st, it, hist = P.solve("pcg", b, u, rtol=1e-8, maxit=500)
            ev[k][2].record(stream)
            its.append(it)
        barrier()
    launches = launch_count() - l0
    applies = (P.fine_applies() - a0) / args.steps - 1
    apply_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1, _ in ev)
    solve_ms = statistics.mean(e1.elapsed_time(e2) for _, e1, e2 in ev)
    step_ms = statistics.mean(e0.elapsed_time(e2) for e0, _, e2 in ev)
    t_apply, value = aggregate_ranks(apply_ms, N, world, dist, dev)
    t_step, _ = aggregate_ranks(step_ms, N, world, dist, dev)
    rel_res = float(hist[-1] / hist[0])

    # ---- end to end through the host-buffer C ABI calls: page-locked x in, y out (apply) and
    # nodal f in, u out (rhs + solve), every copy inside the timed region
    x_host = x.cpu().pin_memory()
    y_host = torch.empty(N, dtype=torch.float64).pin_memory()
    u_host = torch.empty(N, dtype=torch.float64).pin_memory()
    P.apply_host(0, x_host, y_host)
    P.solve_host("pcg", f_host, u_host, rtol=1e-8, maxit=500)
    barrier()
    ta = time.perf_counter()
    for _ in range(args.steps):
        P.apply_host(0, x_host, y_host)
    e2e_apply_ms = (time.perf_counter() - ta) * 1e3 / args.steps
    ts = time.perf_counter()
    for _ in range(args.steps):
        st_h, it_h, _ = P.solve_host("pcg", f_host, u_host, rtol=1e-8, maxit=500)
    e2e_solve_ms = (time.perf_counter() - ts) * 1e3 / args.steps
    barrier()
    _, e2e_value = aggregate_ranks(e2e_apply_ms, N, world, dist, dev)
    e2e_err = float((y_host.to(dev) - y).abs().max() / y.abs().max())
    u_err = float((u_host.to(dev) - u).abs().max() / u.abs().max())

    # ---- roofline of the dominant kernel: the FP64 order-p apply (FP64 pipe)
    (E3, p, _) = P.level_info(0)
    n = p + 1
    E = E3[0] * E3[1] * E3[2]
    v64 = P.level_variants(0)[0]
    flops = E * flop_per_elem(3, n)
    achieved_tf = flops / (apply_ms * 1e-3) / 1e12
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    roof_ms = solve_roofline_ms(P, its[-1], hbm, peak64)
    kern = f"k_apply64<3,{n},{v64}>"
    traffic = APPLY_TRAFFIC.get((kern, E))

    # ---- context blocks (not part of the timed steps)
    mixed = {} if args.host_loop or args.quick else mixed_block(prob, P, b, flush, stream, solve_ms)
    df64 = {} if args.host_loop or args.quick else df64_block(prob, P, b, flush, stream, solve_ms, t_apply, peak64)
    sweep = [] if args.host_loop or args.quick else sweep_block(flush, stream, peak64, orders=((64, 2), (16, 8), (8, 16)))
    c2 = {} if args.host_loop or args.quick else c2_block(flush, stream)
    batched = {} if args.host_loop or args.quick else batched_block(args.batch)
    serving = {} if args.host_loop or args.quick else serve_block(args.requests, args.slots)

    if rank == 0:
        cpu = cpu_baseline(args.hier) if not args.quick else None
        line = {
            "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "hier": args.hier, "global_batch": world, "dof": N,
                       "parallelism": f"replicas{world}",
                       "l2": "flushed before every timed step (256 MB written, then another 256 MB read, so no "
                             "dirty lines remain); the apply's 196.6 MB of FP64 geometric factors also exceed L2",
                       "step": "hmg_apply on the finest level, then hmg_solve (PCG + p-MG) to 1e-8",
                       "solve_loop": "host" if args.host_loop else "graph",
                       "v_cycle": args.prec if args.host_loop else "fp64"},
            "apply_ms": t_apply, "solve_ms": solve_ms, "setup_ms": setup_ms, "iterations": its[-1],
            "final_rel_residual": rel_res,
            "fine_applies_per_solve": applies,
            # per PCG iteration: A p, then a V(3,3) whose pre-smoother starts from zero (2 applies),
            # the restricted residual (1) and the post-smoother (3)
            "fine_applies_model": 7 * its[-1],
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak64, "unit": "TFLOP/s",
                         "frac": achieved_tf / peak64, "traffic": traffic, "kernel": kern,
                         "units_per_launch": E, "flop_per_unit": flop_per_elem(3, n),
                         "traffic_source": TRAFFIC_SOURCE if traffic else None,
                         "note": "FP64 pipe; peak = measured FP64 FMA rate of this GPU (hmg_measure_peak, "
                                 "burst); algorithmic flops 24n^4+15n^3 per element; apply time = hmg_apply "
                                 "(zeroing y + the apply kernel) with CUDA events in the timed steps"},
            "solve_roofline": {"roofline_ms": roof_ms, "measured_ms": solve_ms, "frac": roof_ms / solve_ms,
                               "model": "every apply at max(flops/FP64 peak, bytes/HBM) + vector passes and "
                                        "coarsest GEMV at HBM (HBM peak from MEASURED_PEAKS.json)"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GDOF/s", "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8,
                    "call": "hmg_apply_host (page-locked x -> y)", "ms": e2e_apply_ms, "max_rel_diff_vs_device": e2e_err},
            "e2e_solve": {"ms": e2e_solve_ms, "dof_per_s": N / (e2e_solve_ms * 1e-3), "status": st_h,
                          "iterations": it_h, "call": "hmg_solve_host (page-locked nodal f -> u)",
                          "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8, "max_rel_diff_vs_device": u_err},
            "mixed_precision": mixed, "double_float_operator": df64, "sweep_129cube": sweep,
            "single_solve_16cube_q4": c2,
            "batched_512": batched, "serving": serving,
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    P.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def c2_block(flush, stream):
    """The 16^3 Q4 warped var-coef problem (65^3 = 274,625 DOF, seed 2) with both of its
    hierarchies, FP64 PCG to 1e-8 (median of 10 L2-flushed solves) and its fine apply."""
    import torch

    import synth
    from paper_1402_5938_gb300 import Problem
    out = {"workload": "3D warped var-coef Q4 16^3 (65^3=274,625 DOF), PCG + V(3,3) Chebyshev(3), FP64"}
    for hier in ("p", "h"):
        P = Problem(workload(hier, 16, 4))
        N = P.ndof(0)
        b = torch.zeros(N, dtype=torch.float64, device="cuda")
        P.rhs(torch.from_numpy(synth.nodal_field(synth.SEED_WARPED_VAR3D, N)).cuda(), b)
        u = torch.zeros_like(b)
        t, st, it = timed_solves(P, b, u, flush, stream, 10)
        y = torch.zeros_like(b)
        ta = timed_apply(lambda: P.apply(0, b, y), flush, stream, 20)
        out[hier] = {"solve_ms": t, "iterations": it, "status": st, "levels": P.nlevels(), "apply_ms": ta,
                     "apply_variant": P.level_variants(0)[0],
                     "apply_frac_of_fp64_peak": 4096 * flop_per_elem(3, 5) / (ta * 1e-3) / 1e12 / fp64_peak()}
        if hier == "p":
            out["mixed_precision"] = mixed_block(workload(hier, 16, 4), P, b, flush, stream, t)
        P.close()
    return out


def sweep_block(flush, stream, peak64, orders):
    """Order sweep at 129^3 nodes, same warp and coefficient (seed 3): per order the FP64 apply
    (fraction of the FP64 peak), FP64 PCG + p-MG to 1e-8, and the FP32 / FP16 / BF16 V-cycles."""
    import torch

    import synth
    from paper_1402_5938_gb300 import Problem
    out = []
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    for E, p in orders:
        prob = synth.warped_var3d(E, p, hier="p")
        P64 = Problem(prob)
        N = P64.ndof(0)
        b = torch.zeros(N, dtype=torch.float64, device="cuda")
        P64.rhs(torch.from_numpy(synth.nodal_field(synth.SEED_PSWEEP3D, N)).cuda(), b)
        y = torch.zeros_like(b)
        t64 = timed_apply(lambda: P64.apply(0, b, y), flush, stream, 10)
        u64 = torch.zeros_like(b)
        s64, st, it64 = timed_solves(P64, b, u64, flush, stream, 3)
        n = p + 1
        v64, _ = P64.level_variants(0)
        row = {"mesh": f"{E}^3 Q{p}", "dof": N, "apply_fp64_ms": t64, "apply_fp64_variant": v64,
               "pcg_fp64_ms": s64, "pcg_fp64_iters": it64, "pcg_fp64_status": st}
        if v64 == 4:   # stored dense element matrices: 2 n^6 flops, 8 n^6 bytes per element
            ex_flops, ex_bytes = E ** 3 * 2 * n ** 6, E ** 3 * 8 * n ** 6 + 16 * N
            row.update({"apply_fp64_kernel": "dense element matrices",
                        "apply_fp64_frac_of_fp64_peak": ex_flops / (t64 * 1e-3) / 1e12 / peak64,
                        "apply_fp64_frac_of_hbm": ex_bytes / (t64 * 1e-3) / 1e9 / hbm})
        else:
            row.update({"apply_fp64_kernel": "sum factorization",
                        "apply_fp64_frac_of_fp64_peak": E ** 3 * flop_per_elem(3, n) / (t64 * 1e-3) / 1e12 / peak64})
        for prec, m in mixed_block(prob, P64, b, flush, stream, s64, reps=3).items():
            row[prec] = m
        out.append(row)
        P64.close()
    return out


def run_sweep(args):
    """Order sweep at ~2M DOF (129^3 nodes; (64^3,2), (32^3,4), (16^3,8), (8^3,16)), same warp and
    coefficient: per order the FP64 apply time and the V-cycle operator's time in FP32, FP16 and
    BF16, and FP64 vs mixed-precision PCG + p-MG time to 1e-8, iterations, the mixed solution's
    FP64 residual. One JSON line per order (not the benchmark line)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    flush = L2Flush("cuda")
    for row in sweep_block(flush, torch.cuda.current_stream(), fp64_peak(), ((64, 2), (32, 4), (16, 8), (8, 16))):
        print(json.dumps(dict(row, sweep=row["mesh"])), flush=True)
    return 0


def batched_block(n=512, reps=3):
    """The batched workload: n independent 3D solves (E in 2..12, p in {2,4,6,8}, contrast 10^k,
    k in 0..4) with an FP32 V-cycle inside FP64 PCG, solved by one batch plan (one graph launch per
    batch, one kernel per operation and group), against the same problems solved one at a time with
    the plain FP64 solver. Wall time around each batch solve (synchronized). The same batch again
    with the double-float finest operator (fp64_arith = df64) in every member."""
    import torch

    import synth
    from paper_1402_5938_gb300 import BatchPlan, Problem, launch_count
    dev = torch.device("cuda", 0)
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
    t0 = time.perf_counter()
    plan = BatchPlan(mixed, "pcg", maxit_cap=500)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    groups, kpi = plan.info()
    us = [torch.zeros_like(b) for b in bs]
    plan.solve(bs, us, rtol=1e-8, maxit=500)                              # warm-up
    tb, l0 = [], launch_count()
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        sts, its, _ = plan.solve(bs, us, rtol=1e-8, maxit=500)
        tb.append(time.perf_counter() - t)
    kernels_per_batch = (launch_count() - l0) / reps
    u6 = [torch.zeros_like(b) for b in bs]
    for P, b, u in zip(fp64, bs, u6):                                   # build graphs
        P.solve("pcg", b, u, rtol=1e-8, maxit=500)
    torch.cuda.synchronize()
    l0 = launch_count()
    t = time.perf_counter()
    its6 = []
    for P, b, u in zip(fp64, bs, u6):
        st, it, _ = P.solve("pcg", b, u, rtol=1e-8, maxit=500)
        its6.append(it)
    t_seq = time.perf_counter() - t
    kernels_seq = launch_count() - l0
    diff = max(float(torch.linalg.norm(a - c) / torch.linalg.norm(c)) for a, c in zip(us, u6))
    worst = 0.0
    for P, b, u in zip(fp64, bs, us):
        rr = torch.zeros_like(b)
        P.apply(0, u, rr)
        worst = max(worst, float(torch.linalg.norm(b - rr) / torch.linalg.norm(b)))
    tbm = statistics.median(tb)
    plan.close()
    for P in mixed:
        P.close()
    # the same batch with the double-float finest operator (fp64_arith = df64; p <= 8 here)
    dfs = []
    for i in range(n):
        dfs.append(Problem(dict(synth.batched_problem(i)[0], fp64_arith="df64")))
    plan = BatchPlan(dfs, "pcg", maxit_cap=500)
    groups_df, _ = plan.info()
    ud = [torch.zeros_like(b) for b in bs]
    plan.solve(bs, ud, rtol=1e-8, maxit=500)                              # warm-up
    td = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        sts_d, its_d, _ = plan.solve(bs, ud, rtol=1e-8, maxit=500)
        td.append(time.perf_counter() - t)
    worst_d = 0.0
    for P, b, u in zip(fp64, bs, ud):
        rr = torch.zeros_like(b)
        P.apply(0, u, rr)
        worst_d = max(worst_d, float(torch.linalg.norm(b - rr) / torch.linalg.norm(b)))
    tbd = statistics.median(td)
    plan.close()
    for P in dfs + fp64:
        P.close()
    return {
        "batched": f"{n} solves", "total_dof": sum(dofs), "setup_s_both_sets": setup_s, "plan_build_s": plan_s,
        "groups": groups, "kernels_per_loop_iteration": kpi, "kernels_per_batch": kernels_per_batch,
        "batched_mixed_s": tbm, "batched_solves_per_s": n / tbm, "batched_gdof_per_s": sum(dofs) / tbm / 1e9,
        "fp64_one_at_a_time_s": t_seq, "fp64_solves_per_s": n / t_seq, "fp64_one_at_a_time_kernels": kernels_seq,
        "speedup_vs_fp64_sequential": t_seq / tbm,
        "all_converged": all(s_ == 0 for s_ in sts), "iters_mixed_mean": statistics.mean(its),
        "iters_fp64_mean": statistics.mean(its6), "max_rel_diff_mixed_vs_fp64": diff,
        "worst_fp64_residual_of_mixed": worst,
        "df64": {"note": "the same batch, members built with the double-float finest operator",
                 "groups": groups_df, "batched_s": tbd, "solves_per_s": n / tbd,
                 "speedup_vs_fp64_sequential": t_seq / tbd, "speedup_vs_mixed_batch": tbm / tbd,
                 "all_converged": all(s_ == 0 for s_ in sts_d), "iters_mean": statistics.mean(its_d),
                 "worst_fp64_residual": worst_d}}


def run_batched(args):
    """The batched workload as its own JSON line (see batched_block)."""
    import __graft_entry__
    __graft_entry__.build()
    print(json.dumps(batched_block(args.batch)), flush=True)
    return 0


def serve_block(R=200, slots=8):
    """Serving workload: Poisson arrivals (2,000/s mean) of 2D/3D solves, DOF log-uniform in
    [1e3, 2e6], p uniform in 1..16, all through the continuous-batching server (hmg_server_*):
    the FP32 V-cycle in FP64 PCG with `slots` workers at the specified rate and at half the
    measured saturated rate, and the plain FP64 solver through the same server with one worker
    (one request at a time) and with `slots` workers, on the same arrivals. p50/p99 latency (submit
    to result on the host, setup of each new hierarchy included) and solves/s. Before the timed
    runs, 48 other requests of the stream are served untimed in each precision (kernel loading).
    One more row: the mixed server whose requests also take the double-float finest operator
    (fp64_arith = df64, orders 1-8; higher orders keep the native FP64 one)."""
    import numpy as np

    import synth
    from paper_1402_5938_gb300 import Server, desc_ndof
    reqs = [synth.serving_request(i) for i in range(R)]
    fs = [synth.nodal_field(seed, desc_ndof(prob)) for prob, seed, _ in reqs]
    gaps = np.array([g for _, _, g in reqs])

    def serve(scale, nslots, prec, arith="fp64"):
        srv = Server(0, 160 << 30, nslots)
        arr = np.cumsum(gaps * scale)
        t0 = time.perf_counter()
        tickets = []
        for (prob, _, _), f, a in zip(reqs, fs, arr):
            dt = t0 + a - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(dict(prob, smooth_prec=prec, fp64_arith=arith), f, rtol=1e-8, mode="pcg",
                                      maxit=500))
        lat, ok, done_at, failed, its = [], 0, [], [], []
        for i, ((t, n), a) in enumerate(zip(tickets, arr)):
            st, u, it, res, l = srv.wait(t, n)
            ok += int(st == 0)
            its.append(it)
            if st != 0:
                p = reqs[i][0]
                failed.append({"i": i, "status": st, "iters": it, "dim": p["dim"], "nelem": p["nelem"][0],
                               "order": p["order"], "res": res})
            lat.append(l)
            done_at.append(a + l)
        span = max(done_at)
        srv.close()
        return dict(p50_ms=1e3 * float(np.percentile(lat, 50)), p99_ms=1e3 * float(np.percentile(lat, 99)),
                    solves_per_s=R / span, ok=ok, offered_per_s=R / arr[-1], mean_iterations=float(np.mean(its)),
                    failed=failed, slots=nslots, v_cycle=prec, fp64_arith=arith)

    # warm-up: 48 other requests of the same stream, untimed, so that no timed run pays the
    # one-time loading of kernels on their first launch (each (dimension, order) brings its own)
    for prec, arith in (("fp32", "fp64"), ("fp64", "fp64"), ("fp32", "df64")):
        srv = Server(0, 160 << 30, slots)
        warm = [synth.serving_request(i) for i in range(R, R + 48)]
        for t, n in [srv.submit(dict(p, smooth_prec=prec, fp64_arith=arith), synth.nodal_field(sd, desc_ndof(p)),
                                rtol=1e-8, mode="pcg", maxit=500) for p, sd, _ in warm]:
            srv.wait(t, n)
        srv.close()
    hot = serve(1.0, slots, "fp32")
    cool = serve(max(1.0, (R / gaps.sum()) / (0.5 * hot["solves_per_s"])), slots, "fp32")
    fp64_one = serve(1.0, 1, "fp64")
    fp64_slots = serve(1.0, slots, "fp64")
    hot_df = serve(1.0, slots, "fp32", "df64")
    return {"serve": f"{R} requests, Poisson 2000/s", "mixed_at_2000_per_s": hot, "mixed_below_saturation": cool,
            "mixed_df64_at_2000_per_s": hot_df, "fp64_one_at_a_time": fp64_one, "fp64_same_slots": fp64_slots,
            "mixed_over_fp64_one_at_a_time_solves_per_s": hot["solves_per_s"] / fp64_one["solves_per_s"]}


def run_serve(args):
    """The serving workload as its own JSON line (see serve_block)."""
    import __graft_entry__
    __graft_entry__.build()
    print(json.dumps(serve_block(args.requests, args.slots)), flush=True)
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
                t_fp64 = flops / (fp64_peak() * 1e12)
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
                                     "peak_tflops": fp64_peak(),
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
    finest levels (FP64 hmg_apply, or hmg_apply_f32 with --prec fp32/fp16/bf16) after setup's applies;
    --arith df64: the finest FP64 operator in double-float arithmetic."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1402_5938_gb300 import Problem
    prob = dict(synth.warped_var3d(args.mesh, args.order, hier=args.hier), fp64_arith=args.arith)
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
    ap.add_argument("--quick", action="store_true", help="headline only (no context blocks, no CPU baseline)")
    ap.add_argument("--ref-rows", type=int, default=REF_ROWS_PER_STEP,
                    help="--impl reference: oracle rows of the apply per step")
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
                    help="--profile-apply: precision of the applied operator; --host-loop: of the V-cycle")
    ap.add_argument("--arith", choices=["fp64", "df64"], default="fp64",
                    help="--profile-apply: arithmetic of the finest FP64 operator (df64: double-float)")
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
