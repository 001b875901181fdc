"""The paper's smoother / two-grid spectral study (Sec. 3.2.3 "Comparison of point smoothers",
Figs. 2-3) on the oracle, 961 interior unknowns for p = 1, 4, 16 (2d-const: unit square, mu = 1;
2d-var: warped square, mu = 1 + 1e6 sum cos^2(2 pi x_i)).

The figures start from the error sum_i v_i (v_i the eigenvectors of A) and plot its coefficients
after six smoothing steps and after one two-grid cycle (h-coarsening, exact coarse solve, 3 + 3
steps). Those coefficients depend on the eigensolver's choice of signs, and of bases inside
repeated eigenvalues (the unit square has many), so the pins use what does not: S and T, the
error propagators of six smoothing steps and of the two-grid cycle, written in the eigenbasis.

* 2d-const: every point smoother damps the upper half of the spectrum (||S V_upper||_2 < 1),
  less at higher order; Chebyshev damps a larger part of the spectrum than Jacobi (more singular
  values of S below 0.1); every two-grid cycle converges (spectral radius rho(T) < 1), more
  slowly at higher order.
* 2d-var: Jacobi is worse than on 2d-const, as smoother and in the two-grid cycle; at p = 16 the
  two-grid cycle with Jacobi does not converge (rho(T) > 1) and the one with Chebyshev does.
"""
import numpy as np
import pytest

import synth
from oracle import multigrid


def propagators(kind, p, smoother):
    """(eigenvalues, V^T S V, V^T T V) of the study's problem."""
    H = multigrid.Hierarchy(synth.spectral_problem(kind, p, smoother))
    lam, V = np.linalg.eigh(H.fine.A.toarray())
    n = len(lam)
    zero = np.zeros(n)
    S = np.stack([H.smooth(0, zero, V[:, j].copy(), 6) for j in range(n)], axis=1)
    T = np.stack([H.vcycle(zero, V[:, j].copy()) for j in range(n)], axis=1)
    return lam, V.T @ S, V.T @ T


@pytest.fixture(scope="module")
def study():
    out = {}
    for k in ("2d-const", "2d-var"):
        for p in (1, 4, 16):
            for s in ("jacobi", "cheb"):
                lam, Ms, Mt = propagators(k, p, s)
                n = len(lam)
                out[(k, p, s)] = dict(upper=np.linalg.norm(Ms[:, n // 2:], 2),
                                      damped=int(np.sum(np.linalg.svd(Ms, compute_uv=False) < 0.1)),
                                      rho=float(np.abs(np.linalg.eigvals(Mt)).max()))
    return out


def test_problem_has_961_unknowns_at_every_order():
    for p in (1, 4, 16):
        H = multigrid.Hierarchy(synth.spectral_problem("2d-const", p), arnoldi=False)
        assert H.fine.A.shape == (961, 961)


@pytest.mark.slow
def test_smoothers_damp_the_upper_spectrum_less_at_high_order(study):
    for s in ("jacobi", "cheb"):
        up = [study[("2d-const", p, s)]["upper"] for p in (1, 4, 16)]
        assert max(up) < 1.0, (s, up)
        assert up[0] < up[1] < up[2], (s, up)


@pytest.mark.slow
def test_chebyshev_damps_a_larger_part_of_the_spectrum(study):
    for p in (1, 4, 16):
        assert study[("2d-const", p, "cheb")]["damped"] > study[("2d-const", p, "jacobi")]["damped"], p


@pytest.mark.slow
def test_two_grid_converges_on_2d_const_more_slowly_at_high_order(study):
    for s in ("jacobi", "cheb"):
        rho = [study[("2d-const", p, s)]["rho"] for p in (1, 4, 16)]
        assert max(rho) < 1.0, (s, rho)
        assert rho[0] < rho[1] < rho[2], (s, rho)


@pytest.mark.slow
def test_variable_coefficient_is_harder_for_jacobi(study):
    for p in (1, 4, 16):
        c, v = study[("2d-const", p, "jacobi")], study[("2d-var", p, "jacobi")]
        assert v["upper"] > c["upper"] and v["rho"] > c["rho"], p


@pytest.mark.slow
def test_two_grid_with_jacobi_diverges_on_2d_var_at_order_16(study):
    assert study[("2d-var", 16, "jacobi")]["rho"] > 1.0
    assert study[("2d-var", 16, "cheb")]["rho"] < 1.0
