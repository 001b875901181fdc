"""The Figs. 2-3 spectral study on the GPU: the error coefficients in A's eigenbasis (the
oracle's eigenvectors) after six smoothing steps and after one two-grid cycle equal the oracle's
(1e-9 absolute on coefficients of size <= ~2; the initial ones are all 1), for point, Chebyshev,
l1 and block Jacobi; and the two-grid spectral radius of 2d-var at p = 16 (Jacobi diverges,
Chebyshev converges) equals the oracle's to 1e-8."""
import numpy as np
import pytest

import synth
from oracle import multigrid

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


CASES = [("2d-const", 4, "jacobi"), ("2d-const", 16, "cheb"), ("2d-var", 16, "jacobi"), ("2d-var", 16, "cheb"),
         ("2d-var", 4, "l1jacobi"), ("2d-var", 16, "blockjacobi"), ("2d-var", 1, "cheb")]


@pytest.mark.parametrize("kind,p,smoother", CASES)
def test_spectral_coefficients_match_oracle(hmg, kind, p, smoother):
    prob = synth.spectral_problem(kind, p, smoother)
    H = multigrid.Hierarchy(prob)
    d = H.fine.disc
    lam, V = np.linalg.eigh(H.fine.A.toarray())
    n = len(lam)
    x0 = np.zeros(d.N)
    x0[d.interior] = V @ np.ones(n)
    cs_ref = V.T @ H.smooth(0, np.zeros(n), x0[d.interior].copy(), 6)
    ctg_ref = V.T @ H.vcycle(np.zeros(n), x0[d.interior].copy())
    P = hmg.Problem(prob)
    xs = torch.from_numpy(x0).to(DEV)
    P.smooth(0, torch.zeros_like(xs), xs, 6)
    # two-grid cycle from x0 with b = 0, in the residual form x0 + B(0 - A x0)
    y = torch.zeros_like(xs)
    P.apply(0, torch.from_numpy(x0).to(DEV), y)
    z = torch.zeros_like(xs)
    P.vcycle(-y, z)
    torch.cuda.synchronize()
    cs = V.T @ xs.cpu().numpy()[d.interior]
    ctg = V.T @ (x0 + z.cpu().numpy())[d.interior]
    assert np.abs(cs - cs_ref).max() <= 1e-9
    assert np.abs(ctg - ctg_ref).max() <= 1e-9
    P.close()


@pytest.mark.parametrize("smoother", ["jacobi", "cheb"])
def test_two_grid_spectral_radius_matches_oracle(hmg, smoother):
    prob = synth.spectral_problem("2d-var", 16, smoother)
    H = multigrid.Hierarchy(prob)
    d = H.fine.disc
    lam, V = np.linalg.eigh(H.fine.A.toarray())
    n = len(lam)
    T_ref = np.stack([H.vcycle(np.zeros(n), V[:, j].copy()) for j in range(n)], axis=1)
    P = hmg.Problem(prob)
    T = np.empty((n, n))
    idx = torch.from_numpy(d.interior).to(DEV)
    x = torch.zeros(d.N, dtype=torch.float64, device=DEV)
    y, z = torch.zeros_like(x), torch.zeros_like(x)
    for j in range(n):
        x.zero_()
        x[idx] = torch.from_numpy(V[:, j]).to(DEV)
        P.apply(0, x, y)
        z.zero_()
        P.vcycle(-y, z)
        T[:, j] = (x + z)[idx].cpu().numpy()
    rho = np.abs(np.linalg.eigvals(V.T @ T)).max()
    rho_ref = np.abs(np.linalg.eigvals(V.T @ T_ref)).max()
    assert abs(rho - rho_ref) <= 1e-8 * rho_ref
    assert (rho > 1.0) == (smoother == "jacobi")
    P.close()
