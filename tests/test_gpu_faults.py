"""Failure detection without faulting the GPU: invalid input is refused on the host, a
non-finite right-hand side ends a solve with HMG_ENAN, an unreachable tolerance with
HMG_ENOCONV (solution and history still written), and a bounded device wait that is made to run
out (an mbarrier nothing completes) returns HMG_ETIMEOUT with the context still usable."""
import ctypes

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


@pytest.mark.parametrize("graph", [1, 0])
def test_nan_rhs_and_maxit(hmg, graph):
    P = hmg.Problem(dict(synth.warped_var3d(4, 2, hier="p"), solve_graph=graph))
    N = P.ndof(0)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    P.rhs(torch.from_numpy(synth.nodal_field(1, N)).to(DEV), b)
    bad = b.clone()
    bad[N // 2] = float("nan")
    u = torch.zeros_like(b)
    st, it, h = P.solve("pcg", bad, u, rtol=1e-8, maxit=50)
    assert st == hmg.hmg.HMG_ENAN
    st, it, h = P.solve("pcg", b, u, rtol=1e-30, maxit=3)
    assert st == hmg.hmg.HMG_ENOCONV and it == 3 and len(h) == 4 and h[-1] < h[0]
    st, it, h = P.solve("pcg", b, u, rtol=1e-8, maxit=50)          # the handle still works
    assert st == 0
    P.close()


def test_bounded_wait_gives_up_and_context_survives(hmg):
    out = ctypes.c_int(-1)
    st = hmg.lib().hmg_selftest_bounded_wait(1000, ctypes.byref(out))
    assert st == hmg.hmg.HMG_ETIMEOUT and out.value == 1
    x = torch.ones(16, device=DEV)
    assert float(x.sum()) == 16.0                                    # the context is usable
    P = hmg.Problem(synth.warped_var3d(2, 2, hier="p", n_hlevels=1))
    P.close()


def test_invalid_arguments_are_refused(hmg):
    P = hmg.Problem(synth.warped_var3d(2, 2, hier="p", n_hlevels=1))
    x = torch.zeros(3, dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        P.apply(0, x, x)                                            # too short for the level
    last = P.nlevels() - 1
    y = torch.zeros(P.ndof(last), dtype=torch.float64, device=DEV)
    with pytest.raises(hmg.HmgError):
        P.prolong(last, y, y)                                       # no coarser level
    with pytest.raises(hmg.HmgError):
        hmg.Problem(dict(synth.warped_var3d(2, 2), mu_a=-1.0))      # coefficient not positive
    P.close()


def test_nonblocking_stream_setup_and_solve_match_default_stream(hmg):
    # torch streams are non-blocking: setup's zeroing and uploads must be ordered on the given
    # stream, not on the legacy default stream
    prob = synth.warped_var3d(4, 4, hier="p")
    ref = hmg.Problem(prob)
    N = ref.ndof(0)
    f = torch.from_numpy(synth.nodal_field(3, N)).to(DEV)
    b0 = torch.zeros(N, dtype=torch.float64, device=DEV)
    ref.rhs(f, b0)
    u0 = torch.zeros_like(b0)
    st0, it0, _ = ref.solve("pcg", b0, u0, rtol=1e-8, maxit=100)
    for rep in range(3):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            P = hmg.Problem(prob, stream=s.cuda_stream)
            b = torch.zeros(N, dtype=torch.float64, device=DEV)
            P.rhs(f, b, stream=s.cuda_stream)
            u = torch.zeros_like(b)
            st, it, _ = P.solve("pcg", b, u, rtol=1e-8, maxit=100, stream=s.cuda_stream)
        s.synchronize()
        assert st == 0 and it == it0
        assert float(torch.linalg.norm(b - b0) / torch.linalg.norm(b0)) < 1e-14
        assert float(torch.linalg.norm(u - u0) / torch.linalg.norm(u0)) < 1e-10
        P.close()
    ref.close()
