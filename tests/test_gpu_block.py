"""Element-block Jacobi (the paper's Table 7 block variant) on the GPU against the oracle.

The GPU forms each element's interior block of K_e by sum-factorized unit columns and inverts
it by Gauss-Jordan; the oracle takes the same block out of the assembled CSR matrix and inverts
it with LAPACK. Smoothing and V-cycle results agree to 1e-10 relative: the inverses carry
rounding of about cond(block) * 2^-53, and the blocks here have condition numbers below 1e5.
Solve iteration counts agree within 1, and the Table 7 2d-const rows follow the paper."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import multigrid

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


@pytest.fixture(scope="module")
def hmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1402_5938_gb300 as pkg
    return pkg


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [
    synth.problem(2, (8, 6), 2, warp_amp=0.1, mu_b=1e3, hier="h", n_hlevels=2, smoother="blockjacobi"),
    synth.problem(2, (7, 5), 5, warp_amp=0.1, mu_b=1e3, hier="p", n_hlevels=1, smoother="blockjacobi"),
    synth.problem(2, (4, 4), 8, warp_amp=0.1, mu_b=1e3, hier="h", n_hlevels=2, smoother="blockjacobi"),
    synth.problem(2, (3, 2), 16, hier="p", n_hlevels=1, smoother="blockjacobi"),
    synth.problem(3, (4, 4, 2), 3, warp_amp=0.1, mu_b=1e3, hier="h", n_hlevels=2, smoother="blockjacobi"),
    synth.problem(3, (3, 2, 2), 4, warp_amp=0.1, mu_b=1e3, hier="p", n_hlevels=1, smoother="blockjacobi"),
    synth.problem(3, (2, 2, 2), 6, warp_amp=0.1, mu_b=10.0, hier="h", n_hlevels=2, smoother="blockjacobi"),
]


@pytest.mark.parametrize("prob", CASES, ids=lambda c: f"{c['dim']}d-{c['nelem']}-p{c['order']}-{c['hier']}")
def test_block_smoother_and_vcycle_match_oracle(hmg, prob):
    """Smoothing from a nonzero and from a zero guess on every smoothed level, and the V-cycle."""
    P = hmg.Problem(prob)
    H = multigrid.Hierarchy(prob)
    assert P.nlevels() == len(H.levels)
    for k in range(P.nlevels() - 1):
        d = H.levels[k].disc
        b = synth.uniform_pm1(40 + k, d.N)
        x0 = synth.uniform_pm1(50 + k, d.N)
        b[d.boundary] = 0
        x0[d.boundary] = 0
        xg = _t(x0)
        P.smooth(k, _t(b), xg, 3)
        xz = torch.zeros(d.N, dtype=torch.float64, device=DEV)
        P.smooth(k, _t(b), xz, 2, zero_guess=True)
        torch.cuda.synchronize()
        assert _rel(xg.cpu().numpy()[d.interior], H.smooth(k, b[d.interior], x0[d.interior], 3)) < 1e-10, k
        assert _rel(xz.cpu().numpy()[d.interior], H.smooth(k, b[d.interior], None, 2)) < 1e-10, k
        assert np.all(xg.cpu().numpy()[d.boundary] == 0.0)
    d = H.fine.disc
    r = synth.uniform_pm1(33, d.N)
    r[d.boundary] = 0
    z = torch.zeros(d.N, dtype=torch.float64, device=DEV)
    P.vcycle(_t(r), z)
    torch.cuda.synchronize()
    assert _rel(z.cpu().numpy()[d.interior], H.vcycle(r[d.interior])) < 1e-10
    P.close()


SOLVES = [
    synth.problem(2, (8, 8), 4, warp_amp=0.1, mu_b=1e3, hier="h", n_hlevels=3, smoother="blockjacobi"),
    synth.problem(2, 16, 8, hier="h", n_hlevels=3, smoother="blockjacobi"),
    synth.problem(2, 8, 6, warp_amp=0.1, mu_b=1e3, hier="p", n_hlevels=2, smoother="blockjacobi"),
    synth.problem(3, 4, 4, warp_amp=0.1, mu_b=1e3, hier="p", n_hlevels=2, smoother="blockjacobi"),
    synth.problem(3, (4, 4, 4), 3, warp_amp=0.1, mu_b=1e3, hier="h", n_hlevels=2, smoother="blockjacobi"),
]


@pytest.mark.parametrize("prob", SOLVES, ids=lambda c: f"{c['dim']}d-{c['nelem']}-p{c['order']}-{c['hier']}")
def test_block_solves_match_oracle(hmg, prob):
    """MG and PCG iteration counts within 1 of the oracle's, solutions equal to the accuracy the
    1e-8 residual reduction gives."""
    P = hmg.Problem(prob)
    H = multigrid.Hierarchy(prob)
    d = H.fine.disc
    f = synth.nodal_field(71, d.N)
    b = torch.zeros(d.N, dtype=torch.float64, device=DEV)
    P.rhs(_t(f), b)
    bref = d.rhs(f)
    for mode in ("mg", "pcg"):
        u = torch.zeros_like(b)
        st, it, hist = P.solve(mode, b, u, rtol=1e-8, maxit=400)
        uref, it_ref, _, ok = (H.solve_mg if mode == "mg" else H.solve_pcg)(bref)
        assert st == 0 and ok and abs(it - it_ref) <= 1, (mode, it, it_ref)
        assert _rel(u.cpu().numpy()[d.interior], uref) < 1e-6
    P.close()


def test_block_graph_host_loop_and_batched_agree(hmg):
    prob = synth.problem(2, 8, 6, warp_amp=0.1, mu_b=1e3, hier="h", n_hlevels=2, smoother="blockjacobi")
    Pg = hmg.Problem(dict(prob, solve_graph=1))
    Ph = hmg.Problem(dict(prob, solve_graph=0))
    N = Pg.ndof(0)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    Pg.rhs(_t(synth.nodal_field(72, N)), b)
    ug, uh, ub = (torch.zeros_like(b) for _ in range(3))
    stg, itg, _ = Pg.solve("pcg", b, ug, rtol=1e-8)
    sth, ith, _ = Ph.solve("pcg", b, uh, rtol=1e-8)
    sts, its, _ = hmg.solve_batched([Pg], "pcg", [b], [ub], rtol=1e-8)
    assert stg == sth == sts[0] == 0 and itg == ith == its[0]
    assert _rel(ug.cpu().numpy(), uh.cpu().numpy()) < 1e-12 and _rel(ub.cpu().numpy(), uh.cpu().numpy()) < 1e-12
    Pg.close()
    Ph.close()


def test_block_jacobi_rejected_outside_its_range(hmg):
    """FP64 only, and at most 1000 element-interior unknowns per element (3D p <= 11)."""
    for prob in (dict(synth.problem(2, 4, 4, hier="h", n_hlevels=2, smoother="blockjacobi"), smooth_prec="fp32"),
                 synth.problem(3, 2, 12, hier="p", n_hlevels=1, smoother="blockjacobi")):
        with pytest.raises(Exception):
            hmg.Problem(prob)


def _counts(hmg, p, smoother):
    prob = synth.problem(2, 32, p, hier="h", n_hlevels=3, smoother=smoother, nu_pre=3, nu_post=3)
    P = hmg.Problem(prob)
    N = P.ndof(0)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    P.rhs(_t(synth.nodal_field(7, N)), b)
    out = []
    for mode in ("mg", "pcg"):
        u = torch.zeros_like(b)
        st, it, _ = P.solve(mode, b, u, rtol=1e-8, maxit=1000)
        assert st == 0
        out.append(it)
    P.close()
    return out


def test_table7_block_2d_const(hmg):
    """2d-const 32x32, h-MG V(3,3), omega = 2/3: p = 8 counts equal the oracle's (+-1) and lie
    within 1 of the printed 16 / 8; at p = 8 and 16 block Jacobi needs no more iterations than
    point Jacobi, and the block / point ratios are the paper's within 15 %."""
    gold = GOLDEN["table7_block_2d_const"]
    prob = synth.problem(2, 32, 8, hier="h", n_hlevels=3, smoother="blockjacobi", nu_pre=3, nu_post=3)
    H = multigrid.Hierarchy(prob)
    bref = H.fine.disc.rhs(synth.nodal_field(7, H.fine.disc.N))
    mg_ref, pcg_ref = H.solve_mg(bref)[1], H.solve_pcg(bref)[1]
    mg8, pcg8 = _counts(hmg, 8, "blockjacobi")
    assert abs(mg8 - mg_ref) <= 1 and abs(pcg8 - pcg_ref) <= 1
    assert abs(mg8 - gold["blk"]["MG"]["8"]) <= 1 and abs(pcg8 - gold["blk"]["PCG"]["8"]) <= 1
    for p in (8, 16):
        blk = _counts(hmg, p, "blockjacobi")
        pt = _counts(hmg, p, "jacobi")
        for i, key in enumerate(("MG", "PCG")):
            assert blk[i] <= pt[i], (p, key, blk, pt)
            want = gold["blk"][key][str(p)] / gold["pt"][key][str(p)]
            assert abs(blk[i] / pt[i] - want) <= 0.15 * want, (p, key, blk, pt)
