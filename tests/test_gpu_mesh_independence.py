"""Mesh independence of the multigrid-preconditioned CG iteration count (the paper's Sec. 4.4:
with the coarsest grid fixed at 2 x 2 elements, the count stops changing once the fine mesh is
fine enough), with this library's point smoothers; and the GPU count equals the oracle's (+-1)
on the smaller meshes of the same study.

With Chebyshev / Jacobi smoothing the count is flat for 2d-const at every order and for 2d-var
(mu contrast 1e6) up to order 4; at order 8 on 2d-var it moves between 11 and 15 with the mesh
(the paper's SSOR(2,1) stays at 9), and the oracle gives the same counts there (13 at E = 16,
11 at E = 32), so that cell is checked against the oracle instead of for flatness."""
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


def _count(hmg, prob, seed=11):
    P = hmg.Problem(prob)
    N = P.ndof(0)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    P.rhs(torch.from_numpy(synth.nodal_field(seed, N)).to(DEV), b)
    u = torch.zeros_like(b)
    st, it, _ = P.solve("pcg", b, u, rtol=1e-8, maxit=300)
    P.close()
    assert st == 0
    return it


@pytest.mark.parametrize("kind,order", [("2d-const", 1), ("2d-const", 4), ("2d-const", 8), ("2d-var", 1),
                                        ("2d-var", 2), ("2d-var", 4)])
def test_iterations_independent_of_mesh(hmg, kind, order):
    counts = [_count(hmg, synth.mesh_independence_problem(kind, E, order)) for E in (16, 32, 64, 128)]
    assert max(counts) - min(counts) <= 1, counts


@pytest.mark.parametrize("kind,E,order", [("2d-const", 4, 2), ("2d-const", 8, 2), ("2d-const", 8, 4),
                                          ("2d-var", 4, 2), ("2d-var", 8, 2), ("2d-var", 8, 4), ("2d-var", 16, 8)])
def test_mesh_independence_counts_match_oracle(hmg, kind, E, order):
    from oracle import multigrid
    prob = synth.mesh_independence_problem(kind, E, order)
    H = multigrid.Hierarchy(prob)
    d = H.fine.disc
    _, it_ref, _, ok = H.solve_pcg(d.rhs(synth.nodal_field(11, d.N)))
    assert ok
    assert abs(_count(hmg, prob) - it_ref) <= 1
