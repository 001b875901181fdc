"""hmg_restrict_noalloc: the residual restriction for callers that cannot allocate device
memory, and so cannot create a problem handle (its setup allocates the hierarchy). It keeps
its stencils and intermediate arrays in fixed device storage of the library; its output
must equal that of the handle-based hmg_restrict on the same level pair, on two calls in a
row (the second call reuses the storage the first one left behind), and the oracle's
restriction P^T of Sec. 2.2 Eq. (Pstencil) directly. This file is collected last so that a
run that stops at the first failure has run everything else."""
import numpy as np
import pytest

import synth
from oracle import fem, transfer

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


# (workload, halve_mesh): level 0 -> level 1 of the handle's hierarchy
CASES = [
    (synth.problem(3, (4, 2, 2), 3, warp_amp=0.1, mu_b=1e3, hier="h", n_hlevels=2, smoother="jacobi"), True),
    (synth.problem(3, (2, 2, 2), 8, warp_amp=0.1, mu_b=1e3, hier="p", n_hlevels=1, smoother="jacobi"), False),
    (synth.problem(2, (6, 4), 2, hier="h", n_hlevels=2, smoother="jacobi"), True),
    (synth.problem(2, (3, 5), 16, hier="p", n_hlevels=1, smoother="jacobi"), False),
    (synth.warped_var3d(16, 4, hier="p", smoother="jacobi"), False),   # the 274,625-node level
]


@pytest.mark.parametrize("prob,halve", CASES, ids=lambda c: str(c)[:50])
def test_restrict_noalloc_matches_restrict_on_two_calls(hmg, prob, halve):
    P = hmg.Problem(prob)
    (Ef, pf, Nf), (Ec, pc, Nc) = P.level_info(0), P.level_info(1)
    dim = prob["dim"]
    rf = torch.from_numpy(synth.uniform_pm1(41, Nf)).to(DEV)     # boundary entries nonzero too
    ref = torch.zeros(Nc, dtype=torch.float64, device=DEV)
    P.restrict(0, rf, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for call in range(2):
        rc = torch.full((Nc,), float("nan"), dtype=torch.float64, device=DEV)
        hmg.restrict_noalloc(dim, Ef[:dim], pf, pc, halve, rf, rc)
        torch.cuda.synchronize()
        out = rc.cpu().numpy()
        assert np.all(np.isfinite(out)), f"call {call}: entries left unwritten"
        assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max(), f"call {call}"
    P.close()


# (dim, fine elements, fine order, coarse order, halve): one h- and one p-transfer per dimension
ORACLE_CASES = [(2, (6, 4), 2, 2, True), (2, (3, 5), 6, 3, False), (3, (4, 2, 2), 3, 3, True),
                (3, (2, 3, 2), 4, 2, False)]


@pytest.mark.parametrize("case", ORACLE_CASES, ids=lambda c: str(c))
def test_restrict_noalloc_matches_oracle_transpose(hmg, case):
    dim, E, pf, pc, halve = case
    fine = fem.Discretization(dim, E, pf, warp_amp=0.1)
    coarse = fem.Discretization(dim, tuple(e // 2 for e in E) if halve else E, pc, warp_amp=0.1)
    Pm = transfer.prolongation(fine, coarse)
    rf = synth.uniform_pm1(43, fine.N)
    want = Pm.T @ rf[fine.interior]
    for call in range(2):
        rc = torch.full((coarse.N,), float("nan"), dtype=torch.float64, device=DEV)
        hmg.restrict_noalloc(dim, E, pf, pc, halve, torch.from_numpy(rf).to(DEV), rc)
        torch.cuda.synchronize()
        out = rc.cpu().numpy()
        assert np.all(out[coarse.boundary] == 0.0), f"call {call}"
        assert np.abs(out[coarse.interior] - want).max() <= 1e-13 * np.abs(want).max(), f"call {call}"


def test_restrict_noalloc_rejects_short_buffers(hmg):
    nf, nc = hmg.noalloc_lengths(3, (4, 2, 2), 3, 3, True)
    rf = torch.zeros(nf, dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        hmg.restrict_noalloc(3, (4, 2, 2), 3, 3, True, rf, torch.zeros(nc - 1, dtype=torch.float64, device=DEV))
    with pytest.raises(ValueError):
        hmg.restrict_noalloc(3, (4, 2, 2), 3, 3, True, rf[:-1], torch.zeros(nc, dtype=torch.float64, device=DEV))


def _buffers(hmg, *args):
    nf, nc = hmg.noalloc_lengths(*args)
    return (torch.zeros(nf, dtype=torch.float64, device=DEV), torch.zeros(nc, dtype=torch.float64, device=DEV))


def test_restrict_noalloc_rejects_sizes_beyond_its_storage(hmg):
    args = (3, (2048, 2, 2), 4, 4, True)                                  # 8193 nodes on one axis
    with pytest.raises(hmg.HmgError, match="fine nodes along an axis"):
        hmg.restrict_noalloc(*args, *_buffers(hmg, *args))
    args = (3, (64, 64, 64), 4, 4, True)                                  # 257^3 fine nodes
    with pytest.raises(hmg.HmgError, match="fixed scratch"):
        hmg.restrict_noalloc(*args, *_buffers(hmg, *args))
    args = (3, (3, 2, 2), 2, 2, True)                                     # odd count cannot halve
    with pytest.raises(hmg.HmgError):
        hmg.restrict_noalloc(*args, *_buffers(hmg, *args))
