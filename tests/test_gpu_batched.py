"""Device-side graph solves and batched solves.

* The graph solve (one CUDA graph per solve with a device-side WHILE loop) gives the same
  iteration counts and residual histories as the host-driven loop.
* hmg_solve_batched on uneven problems (batched-workload recipe: E in 2..12, p in {2,4,6,8},
  contrast 10^k, FP32 V-cycle in FP64 PCG) gives, for every problem, the same result as
  solving it alone: same iteration count, solutions equal to 1e-8 relative (the two runs
  differ only in the rounding order of the atomic scatter, which the FP32 V-cycle shows)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def hmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1402_5938_gb300 as pkg
    return pkg


CASES = [
    (synth.warped_var3d(4, 4, hier="h"), "pcg"),
    (synth.warped_var3d(4, 4, hier="p"), "mg"),
    (dict(synth.warped_var3d(4, 4, hier="p"), smooth_prec="fp32"), "pcg"),
    (synth.mms2d_poisson(8, 4), "mg"),
]


@pytest.mark.parametrize("prob,mode", CASES, ids=lambda c: str(c)[:50])
def test_graph_solve_equals_host_loop(hmg, prob, mode):
    Pg = hmg.Problem(dict(prob, solve_graph=1))
    Ph = hmg.Problem(dict(prob, solve_graph=0))
    N = Pg.ndof(0)
    f = torch.from_numpy(synth.nodal_field(9, N)).to(DEV)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    Pg.rhs(f, b)
    ug, uh = torch.zeros_like(b), torch.zeros_like(b)
    a0g, a0h = Pg.fine_applies(), Ph.fine_applies()
    for rep in range(2):                                   # second call replays the same graph
        stg, itg, hg = Pg.solve(mode, b, ug, rtol=1e-8, maxit=200)
    sth, ith, hh = Ph.solve(mode, b, uh, rtol=1e-8, maxit=200)
    assert stg == 0 and sth == 0 and itg == ith
    # FP64: runs differ only in the FP64 atomic-scatter rounding order; with an FP32 V-cycle the
    # preconditioner's own FP32 rounding order (unit roundoff 6e-8) shows in the history
    fp32 = prob.get("smooth_prec") == "fp32"
    sel = hh > 1e-6 * hh[0]                  # below that the scatter rounding order dominates
    assert np.allclose(hg[sel], hh[sel], rtol=1e-5 if fp32 else 1e-9, atol=0)
    assert float(torch.linalg.norm(ug - uh) / torch.linalg.norm(uh)) < (1e-8 if fp32 else 1e-10)
    assert (Pg.fine_applies() - a0g) == 2 * (Ph.fine_applies() - a0h)
    # maxit reached: status and history still written
    st, it, h = Pg.solve(mode, b, ug, rtol=1e-14, maxit=2)
    assert st == hmg.hmg.HMG_ENOCONV and it == 2 and len(h) == 3
    # zero right-hand side: converged at iteration 0
    st, it, h = Pg.solve(mode, torch.zeros_like(b), ug, rtol=1e-8, maxit=10)
    assert st == 0 and it == 0 and float(torch.linalg.norm(ug)) == 0.0
    Pg.close()
    Ph.close()


def test_batched_equals_alone(hmg):
    probs, bs, us = [], [], []
    for i in range(12):
        prob, seed = synth.batched_problem(i)
        P = hmg.Problem(prob)
        N = P.ndof(0)
        f = torch.from_numpy(synth.nodal_field(seed, N)).to(DEV)
        b = torch.zeros(N, dtype=torch.float64, device=DEV)
        P.rhs(f, b)
        probs.append(P)
        bs.append(b)
        us.append(torch.zeros_like(b))
    sts, its, hists = hmg.solve_batched(probs, "pcg", bs, us, rtol=1e-8, maxit=300)
    assert all(s == 0 for s in sts)
    for P, b, u, it, h in zip(probs, bs, us, its, hists):
        u1 = torch.zeros_like(b)
        st1, it1, h1 = P.solve("pcg", b, u1, rtol=1e-8, maxit=300)
        assert st1 == 0 and it1 == it
        assert float(torch.linalg.norm(u - u1) / torch.linalg.norm(u1)) < 1e-8    # FP32 V-cycle
        assert h[-1] <= 1e-8 * h[0]
    for P in probs:
        P.close()


def test_batched_matches_oracle_counts(hmg):
    from oracle import multigrid
    for i in (0, 3):
        prob, seed = synth.batched_problem(i)
        prob64 = dict(prob, smooth_prec="fp64")
        P = hmg.Problem(prob64)
        N = P.ndof(0)
        f = synth.nodal_field(seed, N)
        b = torch.zeros(N, dtype=torch.float64, device=DEV)
        P.rhs(torch.from_numpy(f).to(DEV), b)
        u = torch.zeros_like(b)
        sts, its, _ = hmg.solve_batched([P], "pcg", [b], [u], rtol=1e-8, maxit=300)
        H = multigrid.Hierarchy(prob64)
        _, it_ref, _, ok = H.solve_pcg(H.fine.disc.rhs(f))
        assert sts[0] == 0 and ok and abs(its[0] - it_ref) <= 1
        P.close()


@pytest.mark.parametrize("mode", ["mg", "pcg"])
def test_batched_lockstep_edges(hmg, mode):
    """Mixed batch: ordinary solves, a zero right-hand side (converged at iteration 0) and a
    problem that runs out of iterations; histories agree with solving each problem alone."""
    probs, bs = [], []
    for i in (1, 2, 5):
        prob, seed = synth.batched_problem(i)
        P = hmg.Problem(prob)
        N = P.ndof(0)
        b = torch.zeros(N, dtype=torch.float64, device=DEV)
        P.rhs(torch.from_numpy(synth.nodal_field(seed, N)).to(DEV), b)
        probs.append(P)
        bs.append(b)
    bs[1].zero_()
    us = [torch.full_like(b, 7.0) for b in bs]
    sts, its, hists = hmg.solve_batched(probs, mode, bs, us, rtol=1e-8, maxit=60)
    assert sts[0] == 0 and sts[1] == 0 and its[1] == 0 and float(torch.linalg.norm(us[1])) == 0.0
    for k in (0, 2):
        u1 = torch.zeros_like(bs[k])
        st1, it1, h1 = probs[k].solve(mode, bs[k], u1, rtol=1e-8, maxit=60)
        assert st1 == sts[k] and it1 == its[k] and len(hists[k]) == its[k] + 1
        big = [j for j in range(len(h1)) if h1[j] > 1e-6 * h1[0]]
        assert max(abs(hists[k][j] - h1[j]) / h1[j] for j in big) < 1e-5  # FP32 V-cycle
        assert float(torch.linalg.norm(us[k] - u1) / torch.linalg.norm(u1)) < 1e-8
    # an iteration cap below what problem 0 needs
    cap = max(1, its[0] - 2)
    us = [torch.zeros_like(b) for b in bs]
    sts, its2, hists = hmg.solve_batched(probs, mode, bs, us, rtol=1e-8, maxit=cap)
    assert sts[0] == hmg.hmg.HMG_ENOCONV and its2[0] == cap and len(hists[0]) == cap + 1
    assert sts[1] == 0 and its2[1] == 0
    for P in probs:
        P.close()


def _batch(hmg, idx, **over):
    probs, bs = [], []
    for i in idx:
        prob, seed = synth.batched_problem(i)
        prob = dict(prob, **over)
        P = hmg.Problem(prob)
        N = P.ndof(0)
        b = torch.zeros(N, dtype=torch.float64, device=DEV)
        P.rhs(torch.from_numpy(synth.nodal_field(seed, N)).to(DEV), b)
        probs.append(P)
        bs.append(b)
    return probs, bs


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_batch_plan_groups_and_repeats(hmg, prec):
    """A plan over problems of several orders: one group per hierarchy structure, a bounded number
    of kernels per loop iteration (one launch per operation and group, not per problem), and two
    solves in a row give every problem the iterations and solution of solving it alone."""
    probs, bs = _batch(hmg, range(10), smooth_prec=prec)
    plan = hmg.BatchPlan(probs, "pcg", maxit_cap=300)
    groups, kpi = plan.info()
    orders = {P.level_info(0)[1] for P in probs}
    assert groups == len(orders)
    assert kpi < 150 * groups
    alone = []
    for P, b in zip(probs, bs):
        u1 = torch.zeros_like(b)
        st1, it1, _ = P.solve("pcg", b, u1, rtol=1e-8, maxit=300)
        alone.append((st1, it1, u1))
    tol = 1e-10 if prec == "fp64" else (1e-8 if prec == "fp32" else 1e-6)
    for rep in range(2):
        us = [torch.full_like(b, 3.0) for b in bs]
        sts, its, hists = plan.solve(bs, us, rtol=1e-8, maxit=300)
        for (st1, it1, u1), st, it, u, h in zip(alone, sts, its, us, hists):
            assert st == st1 == 0 and (it == it1 if prec != "bf16" else abs(it - it1) <= 1), (rep, it, it1)
            assert h[-1] <= 1e-8 * h[0]
            assert float(torch.linalg.norm(u - u1) / torch.linalg.norm(u1)) < tol
    plan.close()
    for P in probs:
        P.close()


def test_batch_plan_double_float_operator(hmg):
    """Members built with the double-float finest operator (fp64_arith = df64) form groups of
    their own and run it inside the plan: two solves in a row give every member the iterations and
    solution of solving it alone, and its true FP64 residual (native FP64 operator) meets 1e-8."""
    probs, bs = [], []
    for i in range(8):
        prob, seed = synth.batched_problem(i)
        prob = dict(prob, smooth_prec="fp32", fp64_arith="df64" if i % 2 == 0 else "fp64")
        P = hmg.Problem(prob)
        assert (P.level_variants(0)[0] == 7) == (i % 2 == 0)
        N = P.ndof(0)
        b = torch.zeros(N, dtype=torch.float64, device=DEV)
        P.rhs(torch.from_numpy(synth.nodal_field(seed, N)).to(DEV), b)
        probs.append(P)
        bs.append(b)
    plan = hmg.BatchPlan(probs, "pcg", maxit_cap=300)
    groups, _ = plan.info()
    assert groups == len({(P.level_info(0)[1], P.level_variants(0)[0] == 7) for P in probs})
    alone = []
    for P, b in zip(probs, bs):
        u1 = torch.zeros_like(b)
        st1, it1, _ = P.solve("pcg", b, u1, rtol=1e-8, maxit=300)
        alone.append((st1, it1, u1))
    for rep in range(2):
        us = [torch.full_like(b, 3.0) for b in bs]
        sts, its, hists = plan.solve(bs, us, rtol=1e-8, maxit=300)
        for i, ((st1, it1, u1), st, it, u) in enumerate(zip(alone, sts, its, us)):
            assert st == st1 == 0 and it == it1, (rep, i, it, it1)
            assert float(torch.linalg.norm(u - u1) / torch.linalg.norm(u1)) < 1e-8
    for i, (P, b, u) in enumerate(zip(probs, bs, us)):
        if i % 2:
            continue
        ref = hmg.Problem(dict(synth.batched_problem(i)[0], smooth_prec="fp32"))
        r = torch.zeros_like(b)
        ref.apply(0, u, r)
        assert float(torch.linalg.norm(b - r) / torch.linalg.norm(b)) <= 1.1e-8
        ref.close()
    plan.close()
    for P in probs:
        P.close()


def test_batch_plan_mg_mode_2d_and_3d(hmg):
    """MG iteration in a plan that mixes 2D and 3D problems (separate groups)."""
    probs, bs = [], []
    for prob in (synth.mms2d_poisson(8, 4), synth.warped_var3d(4, 2, hier="p", n_hlevels=2),
                 synth.problem(2, 12, 3, warp_amp=0.1, mu_b=1e3, hier="h", n_hlevels=2)):
        P = hmg.Problem(prob)
        N = P.ndof(0)
        b = torch.zeros(N, dtype=torch.float64, device=DEV)
        P.rhs(torch.from_numpy(synth.nodal_field(13, N)).to(DEV), b)
        probs.append(P)
        bs.append(b)
    plan = hmg.BatchPlan(probs, "mg", maxit_cap=100)
    us = [torch.zeros_like(b) for b in bs]
    sts, its, hists = plan.solve(bs, us, rtol=1e-8, maxit=100)
    for P, b, u, st, it in zip(probs, bs, us, sts, its):
        u1 = torch.zeros_like(b)
        st1, it1, _ = P.solve("mg", b, u1, rtol=1e-8, maxit=100)
        assert st == st1 == 0 and it == it1
        assert float(torch.linalg.norm(u - u1) / torch.linalg.norm(u1)) < 1e-10
    plan.close()
    for P in probs:
        P.close()


def test_batched_block_jacobi_falls_back_to_lockstep(hmg):
    """Element-block Jacobi has no grouped form: a plan refuses it, hmg_solve_batched still solves it."""
    prob = synth.problem(2, 8, 4, hier="h", n_hlevels=2, smoother="blockjacobi")
    P = hmg.Problem(prob)
    N = P.ndof(0)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    P.rhs(torch.from_numpy(synth.nodal_field(14, N)).to(DEV), b)
    with pytest.raises(hmg.HmgError):
        hmg.BatchPlan([P], "pcg")
    u = torch.zeros_like(b)
    sts, its, _ = hmg.solve_batched([P], "pcg", [b], [u], rtol=1e-8, maxit=100)
    u1 = torch.zeros_like(b)
    st1, it1, _ = P.solve("pcg", b, u1, rtol=1e-8, maxit=100)
    assert sts[0] == st1 == 0 and its[0] == it1
    P.close()
