"""Pins of the oracle's prolongation P_ij = phi_j^coarse(p_i) (Sec. 2.2, Eq. Pstencil)."""
import numpy as np
import pytest

from oracle import fem, transfer


def _pairs():
    # (fine, coarse) level pairs: h-coarsening (same p, half the mesh) and p-coarsening
    return [
        (fem.Discretization(2, 4, 3), fem.Discretization(2, 2, 3)),
        (fem.Discretization(2, 2, 4), fem.Discretization(2, 2, 2)),
        (fem.Discretization(2, 2, 16), fem.Discretization(2, 2, 8)),
        (fem.Discretization(3, 2, 2), fem.Discretization(3, 1, 2)),
        (fem.Discretization(3, 2, 4), fem.Discretization(3, 2, 2)),
        (fem.Discretization(2, (4, 2), 2, warp_amp=0.1), fem.Discretization(2, (2, 1), 2, warp_amp=0.1)),
    ]


@pytest.mark.parametrize("pair", range(6))
def test_prolongation_reproduces_coarse_polynomials(pair):
    fine, coarse = _pairs()[pair]
    P = transfer.prolongation(fine, coarse, interior=False)
    # a polynomial of coordinate degree <= p_c per direction (in reference coordinates)
    # lies in the coarse space: interpolate on coarse nodes, prolongate, compare with
    # the interpolant on the fine nodes.
    rng = np.random.default_rng(pair)
    pc = coarse.p
    coefs = [rng.standard_normal(pc + 1) for _ in range(fine.dim)]

    def poly(X):
        return np.prod([np.polynomial.polynomial.polyval(X[:, k], coefs[k]) for k in range(fine.dim)], axis=0)

    vc = poly(coarse.reference_coords())
    vf = poly(fine.reference_coords())
    assert np.allclose(P @ vc, vf, atol=1e-11)
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-13)


def test_prolongation_injects_at_coinciding_nodes():
    fine, coarse = fem.Discretization(2, 4, 2), fem.Discretization(2, 2, 2)
    P = transfer.prolongation(fine, coarse, interior=False).toarray()
    Xf, Xc = fine.reference_coords(), coarse.reference_coords()
    for j, xc in enumerate(Xc):
        i = np.flatnonzero(np.all(np.abs(Xf - xc) < 1e-14, axis=1))
        assert len(i) == 1
        assert P[i[0], j] == 1.0 and np.count_nonzero(P[i[0]]) == 1


@pytest.mark.parametrize("dim,Ef,pf,Ec,pc", [(2, 4, 2, 2, 2), (2, 2, 4, 2, 2), (2, 2, 8, 2, 4),
                                             (3, 2, 2, 1, 2), (3, 2, 4, 2, 2), (2, 4, 1, 2, 1)])
def test_galerkin_identity_on_affine_constant_coefficient(dim, Ef, pf, Ec, pc):
    # mu = const on affine elements: quadrature is exact on both levels, so the
    # rediscretized coarse operator equals P^T A_f P (nested conforming spaces).
    fine = fem.Discretization(dim, Ef, pf, mu_a=2.5)
    coarse = fem.Discretization(dim, Ec, pc, mu_a=2.5)
    P = transfer.prolongation(fine, coarse)
    Ag = (P.T @ fine.stiffness() @ P).toarray()
    Ac = coarse.stiffness().toarray()
    assert np.max(np.abs(Ag - Ac)) <= 1e-12 * np.max(np.abs(Ac))


def test_rediscretized_coarse_differs_from_galerkin_with_variable_mu():
    # With mu varying, the rediscretized operator is not the Galerkin one: this checks
    # that the hierarchy really evaluates mu at each level's own quadrature points.
    fine = fem.Discretization(2, 4, 2, mu_a=1.0, mu_b=1e3)
    coarse = fem.Discretization(2, 2, 2, mu_a=1.0, mu_b=1e3)
    P = transfer.prolongation(fine, coarse)
    Ag = (P.T @ fine.stiffness() @ P).toarray()
    Ac = coarse.stiffness().toarray()
    assert np.max(np.abs(Ag - Ac)) > 1e-3 * np.max(np.abs(Ac))
