"""Solve server (continuous batching): every request's result is the same whether it runs alone
or in a mix that overlaps on the device, the hierarchy cache serves repeated problems, the
memory budget is enforced (with eviction), and the byte estimate used for admission bounds the
real allocation."""
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


def _mix():
    reqs = [
        (synth.warped_var3d(4, 4, hier="p"), 11),
        (synth.warped_var3d(4, 2, hier="h", n_hlevels=2), 12),
        (synth.mms2d_poisson(8, 4), 13),
        (synth.problem(2, 6, 8, warp_amp=0.1, mu_b=1e3, hier="p", n_hlevels=2), 14),
        (dict(synth.warped_var3d(4, 8, hier="p", n_hlevels=1), smooth_prec="fp32"), 15),
        (synth.problem(3, 2, 16, warp_amp=0.1, mu_b=10.0, hier="p", n_hlevels=1), 16),
        (synth.problem(3, 6, 3, warp_amp=0.1, mu_b=1e2, hier="p", n_hlevels=1, smoother="jacobi"), 17),
    ]
    reqs += [(reqs[0][0], 21), (reqs[2][0], 22), (reqs[4][0], 23)]    # repeated problems, new data
    return reqs


def _alone(hmg, prob, f):
    P = hmg.Problem(prob)
    N = P.ndof(0)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    P.rhs(torch.from_numpy(f).to(DEV), b)
    u = torch.zeros_like(b)
    st, it, h = P.solve("pcg", b, u, rtol=1e-8, maxit=500)
    P.close()
    return st, it, u.cpu().numpy()


@pytest.mark.parametrize("budget_gb,slots", [(8, 4), (0.25, 3)])
def test_server_results_equal_alone(hmg, budget_gb, slots):
    srv = hmg.Server(0, int(budget_gb * (1 << 30)), slots)
    reqs = _mix()
    tickets = []
    for prob, seed in reqs:
        f = synth.nodal_field(seed, hmg.desc_ndof(prob))
        tickets.append((srv.submit(prob, f, rtol=1e-8, mode="pcg", maxit=500), prob, f))
    for (t, n), prob, f in tickets:
        st, u, it, res, lat = srv.wait(t, n)
        st1, it1, u1 = _alone(hmg, prob, f)
        assert st == 0 and st1 == 0
        assert it == it1
        tol = 1e-8 if prob.get("smooth_prec") == "fp32" else 1e-10
        assert np.linalg.norm(u - u1) <= tol * np.linalg.norm(u1)
        assert 0 < res <= 1e-8 and lat > 0
    s = srv.stats()
    assert s["completed"] == len(reqs)
    if budget_gb >= 1:
        assert s["cache_hits"] >= 1            # repeated problems reuse resident hierarchies
    assert s["resident_bytes"] <= budget_gb * (1 << 30)
    srv.close()


def test_server_rejects_requests_beyond_budget(hmg):
    srv = hmg.Server(0, 64 << 20, 2)
    prob = synth.warped_var3d(16, 4, hier="p")
    with pytest.raises(hmg.HmgError):
        srv.submit(prob, np.zeros(hmg.desc_ndof(prob)))
    srv.close()


def test_estimate_bounds_allocation(hmg):
    for prob in (synth.warped_var3d(8, 4, hier="h"), synth.warped_var3d(8, 4, hier="p"),
                 dict(synth.warped_var3d(4, 8, hier="p"), smooth_prec="fp32"), synth.mms2d_poisson(8, 4),
                 dict(synth.warped_var3d(8, 4, hier="p"), smooth_prec="fp32", fp64_arith="df64"),
                 dict(synth.warped_var3d(4, 6, hier="p"), smoother="blockjacobi"),
                 synth.problem(2, 8, 8, hier="h", smoother="l1jacobi")):
        res, peak = hmg.estimate_bytes(prob)
        P = hmg.Problem(prob)
        actual = P.device_bytes()
        assert actual <= res <= 1.3 * actual + (1 << 20)
        assert peak >= res
        P.close()
