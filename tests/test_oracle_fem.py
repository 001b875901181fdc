"""Pins of the oracle's discretization (Sec. 2.1, 2.3): textbook stencils, brute-force
quadrature, operator invariants, an exact patch test and manufactured-solution
convergence at the rate O(h^(p+1))."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem


def test_q1_square_element_matrix_textbook():
    # Bilinear element on the unit square, mu = 1: diagonal 2/3, edge neighbours -1/6,
    # the opposite corner -1/3 (local order (0,0),(1,0),(0,1),(1,1)).
    d = fem.Discretization(2, 1, 1)
    K = d.element_matrices([0])[0]
    ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    assert np.allclose(K, ref, atol=1e-15)


def test_q1_assembled_stencils_2d_3d():
    d2 = fem.Discretization(2, 4, 1)
    A2 = d2.assemble().toarray()
    g = 2 * 5 + 2                                   # centre node of the 5x5 grid
    row = A2[g].reshape(5, 5)[1:4, 1:4]
    # bilinear Laplacian 9-point stencil: centre 8/3, all eight neighbours -1/3
    assert np.isclose(row[1, 1], 8 / 3)
    nb = np.delete(row.ravel(), 4)
    assert np.allclose(nb, -1 / 3)
    assert abs(A2[g].sum()) < 1e-14
    # 3D trilinear Laplacian on a uniform grid (spacing h = 1/4): centre 8h/3, faces 0,
    # edges -h/6, corners -h/12.
    d3 = fem.Discretization(3, 4, 1)
    A3 = d3.assemble()
    g = (2 * 5 + 2) * 5 + 2
    row = A3[g].toarray().reshape(5, 5, 5)[1:4, 1:4, 1:4]
    h = 0.25
    cnt = np.abs(np.indices((3, 3, 3)) - 1).sum(axis=0)
    assert np.isclose(row[1, 1, 1], 8 * h / 3)
    assert np.allclose(row[cnt == 1], 0.0, atol=1e-15)
    assert np.allclose(row[cnt == 2], -h / 6)
    assert np.allclose(row[cnt == 3], -h / 12)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 3), (2, 6), (3, 2), (3, 3)])
def test_affine_elements_exact_with_p_plus_1_gauss_points(dim, p):
    # Rectangular (affine) elements, mu = 1: q = p+1 integrates the stiffness exactly, so a
    # brute-force rule with q = p+3 must give the same element matrices.
    d = fem.Discretization(dim, (2, 3, 1)[:dim], p)
    els = np.arange(d.n_elem)
    assert np.allclose(d.element_matrices(els), d.element_matrices(els, q=p + 3), atol=1e-12)
    assert np.allclose(d.element_matrices(els, mass=True),
                       d.element_matrices(els, q=p + 3, mass=True), atol=1e-14)


@pytest.mark.parametrize("dim,E,p", [(2, 3, 4), (3, 2, 3)])
def test_operator_symmetric_neumann_kernel_and_spd(dim, E, p):
    d = fem.Discretization(dim, E, p, warp_amp=0.1, mu_a=1.0, mu_b=1e3, mu_k=2.0)
    Af = d.assemble()
    scale = abs(Af).max()
    assert abs(Af - Af.T).max() <= 1e-14 * scale
    # pure-Neumann operator annihilates constants
    assert np.max(np.abs(Af @ np.ones(d.N))) <= 1e-12 * scale
    A = d.stiffness().toarray()
    np.linalg.cholesky(A)               # positive definite on the interior


def test_patch_test_linear_function_2d_warped():
    # mu = 1: a linear function of the PHYSICAL coordinates lies in the isoparametric
    # space, and a(x_k, phi_i) = 0 for interior i (Laplace of a linear function), exactly
    # in 2D with q = p+1 Gauss points. A transposed Jacobian breaks this.
    for p in (1, 2, 4):
        d = fem.Discretization(2, 3, p, warp_amp=0.1)
        Af = d.assemble()
        X = d.node_coords()
        for k in range(2):
            r = (Af @ X[:, k])[d.interior]
            assert np.max(np.abs(r)) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_mapped_domain_measure(dim):
    # The warp fixes the boundary, so the mapped domain is still the unit square/cube.
    d = fem.Discretization(dim, 3, 3, warp_amp=0.1)
    Phi, dPhi, W = d.basis_tables()
    _, _, detJ = d.element_geometry(np.arange(d.n_elem))
    vol = np.sum(W[None, :] * detJ)
    assert np.all(detJ > 0)
    assert abs(vol - 1.0) < (1e-13 if dim == 2 else 1e-6)


def _mms_error(dim, E, p, warp, mu_b):
    """L2 error of the Galerkin solution for u = prod sin(pi x_i) with
    mu = 1 + mu_b sum cos^2(2 pi x_i) (f = -div(mu grad u) written out by hand)."""
    d = fem.Discretization(dim, E, p, warp_amp=warp, mu_a=1.0, mu_b=mu_b, mu_k=2.0)
    k = 2.0

    def u_ex(x):
        return np.prod(np.sin(np.pi * x), axis=1)

    def f_ex(x):
        mu = 1.0 + mu_b * np.sum(np.cos(k * np.pi * x) ** 2, axis=1)
        f = dim * np.pi ** 2 * mu * u_ex(x)
        for i in range(dim):
            # -dmu/dx_i * du/dx_i, dmu/dx_i = -mu_b k pi sin(2 k pi x_i)
            du = np.pi * np.cos(np.pi * x[:, i]) * np.prod(
                np.sin(np.pi * np.delete(x, i, axis=1)), axis=1)
            f += mu_b * k * np.pi * np.sin(2 * k * np.pi * x[:, i]) * du
        return f

    X = d.node_coords()
    b = d.rhs(f_ex(X))
    u = spla.spsolve(d.stiffness().tocsc(), b)
    uf = d.to_full(u)
    tables = d.basis_tables()
    Phi, _, W = tables
    els = np.arange(d.n_elem)
    xq, _, detJ = d.element_geometry(els, tables)
    uq = np.einsum("qa,ea->eq", Phi, uf[d.element_nodes(els)])
    err = uq - u_ex(xq.reshape(-1, dim)).reshape(uq.shape)
    return np.sqrt(np.sum(W[None, :] * detJ * err ** 2))


@pytest.mark.parametrize("dim,p,Es", [(2, 1, (16, 32)), (2, 2, (32, 64)), (2, 3, (16, 32)),
                                      (2, 4, (16, 32)), (3, 1, (8, 16)), (3, 2, (4, 8))])
def test_mms_convergence_rate_p_plus_1_warped_variable_mu(dim, p, Es):
    # Asymptotic L2 rate p+1; on the coarser pairs the rate still approaches p+1 from
    # above (pre-asymptotic), so only the lower side is tight. A wrong geometric factor,
    # quadrature weight or coefficient evaluation stalls the rate near 0.
    errs = [_mms_error(dim, E, p, 0.1, 1.0) for E in Es]
    rate = np.log(errs[-2] / errs[-1]) / np.log(Es[-1] / Es[-2])
    assert p + 1 - 0.3 < rate < p + 1 + 2.5, (errs, rate)
    assert errs[-1] < 1e-2


def test_apply_rows_equals_assembled_rows():
    d = fem.Discretization(3, 2, 3, warp_amp=0.1, mu_a=1.0, mu_b=1e3)
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, d.N)
    x[d.boundary] = 0
    rows = d.interior[rng.choice(d.n_interior, 12, replace=False)]
    ref = (d.assemble() @ x)[rows]
    assert np.allclose(d.apply_rows(x, rows), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("dim,E,p", [(2, (3, 2), 5), (3, (2, 2, 1), 3), (3, (1, 1, 1), 11)])
def test_diag_rows_equals_assembled_diagonal(dim, E, p):
    # the weak form with u_h = phi_i (the GPU diagonal's reference where A cannot be assembled)
    # against the diagonal of the assembled element matrices; p = 11 in 3D is one of the sizes
    # the GPU tests check only by sampled rows
    d = fem.Discretization(dim, E, p, warp_amp=0.1, mu_a=1.0, mu_b=1e3)
    rng = np.random.default_rng(4)
    rows = d.interior[rng.choice(d.n_interior, min(10, d.n_interior), replace=False)]
    ref = d.assemble().diagonal()[rows]
    got = d.diag_rows(rows)
    assert np.all(ref > 0)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.all(d.diag_rows(np.flatnonzero(d.boundary)[:3]) == 0.0)


@pytest.mark.parametrize("dim,E,p", [(2, (3, 2), 5), (3, (2, 1, 2), 4), (3, (1, 1, 1), 11)])
def test_mass_rows_equals_assembled_mass(dim, E, p):
    d = fem.Discretization(dim, E, p, warp_amp=0.1, mu_a=1.0, mu_b=1e3)
    rng = np.random.default_rng(5)
    f = rng.uniform(-1, 1, d.N)                      # all N nodal values, boundary included
    rows = d.interior[rng.choice(d.n_interior, min(10, d.n_interior), replace=False)]
    ref = (d.assemble(mass=True) @ f)[rows]
    assert np.abs(d.mass_rows(f, rows) - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("dim,E,p", [(2, (4, 3), 3), (3, (2, 3, 2), 2), (3, (2, 1, 1), 6)])
def test_mass_rows_of_one_are_gll_weights(dim, E, p):
    # On the affine unit square/cube, (M 1)_i = int phi_i; the Lagrange basis on the p+1 GLL
    # nodes of an interval integrates to the GLL quadrature weights (that rule is exact to degree
    # 2p-1 >= p), so int phi_i is the product over axes of the assembled 1D GLL weights of node
    # i's index: closed forms independent of the oracle's quadrature and element tables.
    from oracle import basis
    d = fem.Discretization(dim, E, p)
    r = basis.gll_nodes(p)
    # 1D GLL weights on [0,1] from their definition w_j = 2 / (p (p+1) P_p(x_j)^2) on [-1,1]
    x = 2 * r - 1
    Pp = np.polynomial.legendre.legval(x, [0] * p + [1])
    w = 1.0 / (p * (p + 1) * Pp ** 2)                # halved for [0,1]
    assert np.isclose(w.sum(), 1.0)
    wax = []
    for ax in range(dim):
        v = np.zeros(d.Nn[ax])
        for e in range(d.E[ax]):
            v[e * p:e * p + p + 1] += w / d.E[ax]
        wax.append(v)
    rows = d.interior[:: max(1, d.n_interior // 15)]
    ref = np.ones(len(rows))
    for ax in range(dim):
        ref *= wax[ax][d.node_axis_index[ax][rows]]
    assert np.abs(d.mass_rows(np.ones(d.N), rows) - ref).max() <= 1e-14


# ---- user-given geometry (node_xyz) and coefficient (mu_fn) -------------------------------

def _poly_map(X):
    """A smooth polynomial map of [0,1]^d of degree <= 3 per coordinate (fixes the boundary)."""
    s = np.prod(X * (1.0 - X), axis=1)
    return X + 0.5 * s[:, None] * (1.0 + X[:, :1])


@pytest.mark.parametrize("dim,E,p", [(2, (3, 2), 3), (3, (2, 2, 1), 3), (2, (2, 3), 4)])
def test_map_points_reproduces_polynomial_maps(dim, E, p):
    """Isoparametric interpolation of a map of degree <= p is exact (Sec. 2.3 geometry):
    map_points at arbitrary reference points equals the map itself."""
    ref = fem.Discretization(dim, E, p)
    d = fem.Discretization(dim, E, p, node_xyz=_poly_map(ref.reference_coords()).T)
    pts = np.random.default_rng(3).uniform(0, 1, (200, dim))
    pts[:5] = 0.5                                   # on element faces (either element is fine)
    assert np.abs(d.map_points(pts) - _poly_map(pts)).max() < 1e-13
    plain = fem.Discretization(dim, E, p)
    assert np.abs(plain.map_points(pts) - pts).max() < 1e-14


def test_given_coordinates_and_coefficient_reproduce_the_built_in_ones():
    """node_xyz = the warp at the nodes and mu_fn = the cos^2 formula give the built-in operator
    exactly; a constant mu_fn = c scales the mu = 1 operator by c."""
    d0 = fem.Discretization(2, (3, 2), 3, warp_amp=0.1, mu_b=1e3)
    xyz = d0.node_coords().T
    d1 = fem.Discretization(2, (3, 2), 3, node_xyz=xyz,
                            mu_fn=lambda x: 1.0 + 1e3 * np.sum(np.cos(2.0 * np.pi * x) ** 2, axis=0))
    assert abs(d1.stiffness() - d0.stiffness()).max() == 0.0
    one = fem.Discretization(2, (3, 2), 3, node_xyz=xyz)
    three = fem.Discretization(2, (3, 2), 3, node_xyz=xyz, mu_fn=lambda x: np.full(x.shape[1], 3.0))
    assert abs(three.stiffness() - 3.0 * one.stiffness()).max() <= 1e-14 * abs(one.stiffness()).max()


def test_hierarchy_coarse_levels_use_the_finest_map():
    """With given coordinates, a coarser level's nodes are the finest map at its reference
    nodes: exact for a polynomial map the finest order reproduces (p = 4, degree 3)."""
    import synth
    from oracle import multigrid
    prob = synth.problem(2, 8, 4, hier="p", n_hlevels=2)
    fine = fem.Discretization(2, 8, 4)
    prob = dict(prob, node_xyz=_poly_map(fine.reference_coords()).T)
    H = multigrid.Hierarchy(prob, arnoldi=False)
    for L in H.levels[1:]:
        d = L.disc
        assert np.abs(d.node_coords() - _poly_map(d.reference_coords())).max() < 1e-13
