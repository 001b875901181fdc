"""Pins of the oracle's 1D basis ingredients (Sec. 2.3, Fig. 1) against closed forms."""
import json
import os

import numpy as np
import pytest

from oracle import basis

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def test_gll_p4_matches_fig1():
    # Fig. 1 prints the p=4 LGL nodes on [0,1]; the closed form is (1 -+ sqrt(3/7))/2.
    r = basis.gll_nodes(4)
    assert np.allclose(r, GOLDEN["fig1_gll_p4"]["nodes"], atol=5e-5)
    s = np.sqrt(3.0 / 7.0)
    assert np.allclose(r, [0, (1 - s) / 2, 0.5, (1 + s) / 2, 1], atol=1e-15)


@pytest.mark.parametrize("p,expected", [
    (1, [0.0, 1.0]),
    (2, [0.0, 0.5, 1.0]),
    (3, [0.0, (1 - 1 / np.sqrt(5)) / 2, (1 + 1 / np.sqrt(5)) / 2, 1.0]),
])
def test_gll_closed_forms(p, expected):
    assert np.allclose(basis.gll_nodes(p), expected, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 17))
def test_gll_are_roots_of_legendre_derivative(p):
    r = basis.gll_nodes(p)
    assert len(r) == p + 1 and r[0] == 0.0 and r[-1] == 1.0
    assert np.all(np.diff(r) > 0)
    assert np.allclose(r + r[::-1], 1.0, atol=1e-15)
    if p > 1:
        # Independent check with numpy's Legendre class: P_p'(2r-1) = 0 at interior nodes.
        dP = np.polynomial.legendre.Legendre.basis(p).deriv()
        assert np.max(np.abs(dP(2 * r[1:-1] - 1))) < 1e-10 * p * p


@pytest.mark.parametrize("q", range(1, 18))
def test_gauss_rule_exact_to_degree_2q_minus_1(q):
    x, w = basis.gauss_rule(q)
    for k in range(2 * q):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-14
    # Degree 2q: the Gauss error term on [0,1] is (q!)^4 / ((2q+1) ((2q)!)^3) * g^(2q), i.e.
    # (q!)^4 / ((2q+1) ((2q)!)^2) for g = t^(2q) (checked where it exceeds rounding).
    from math import factorial
    E = factorial(q) ** 4 / ((2 * q + 1) * factorial(2 * q) ** 2)
    if E > 1e-10:
        err = 1.0 / (2 * q + 1) - np.dot(w, x ** (2 * q))
        assert abs(err / E - 1.0) < 1e-4
    ref_x, ref_w = np.polynomial.legendre.leggauss(q)
    assert np.allclose(x, (ref_x + 1) / 2, atol=1e-15)
    assert np.allclose(w, ref_w / 2, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 4, 8, 16])
def test_lagrange_cardinal_partition_and_polynomial_reproduction(p):
    r = basis.gll_nodes(p)
    assert np.allclose(basis.lagrange_values(r, r), np.eye(p + 1), atol=1e-14)
    x = np.linspace(0, 1, 37)
    L = basis.lagrange_values(r, x)
    dL = basis.lagrange_derivatives(r, x)
    assert np.allclose(L.sum(axis=1), 1.0, atol=1e-12)
    assert np.allclose(dL.sum(axis=1), 0.0, atol=1e-9 * p * p)
    rng = np.random.default_rng(p)
    c = rng.standard_normal(p + 1)
    poly = np.polynomial.Polynomial(c)
    assert np.allclose(L @ poly(r), poly(x), atol=1e-11)
    assert np.allclose(dL @ poly(r), poly.deriv()(x), atol=1e-8 * p ** 2)


@pytest.mark.parametrize("p", range(1, 17))
def test_1d_tables_are_centro_symmetric(p):
    """The GLL nodes and the Gauss points are symmetric about the element's centre, so the
    interpolation table B[q][a] = l_a(g_q) is centro-symmetric and the collocated Gauss derivative
    D[q][s] = l^G_s'(g_q) skew-centro-symmetric: A[n-1-i][n-1-j] = +-A[i][j]. The even/odd line
    products of the pencil form rest on this; the half-size products of sums and differences then
    reproduce A x (checked here on seeded vectors for B, D and their transposes)."""
    r = basis.gll_nodes(p)
    g, _ = basis.gauss_rule(p + 1)
    n = p + 1
    B = basis.lagrange_values(r, g)            # [q][a]
    D = basis.lagrange_derivatives(g, g)       # [q][s]
    assert np.allclose(B[::-1, ::-1], B, atol=1e-13 * np.abs(B).max())
    assert np.allclose(D[::-1, ::-1], -D, atol=1e-13 * np.abs(D).max())
    rng = np.random.default_rng(p)
    h = n // 2
    for A, sgn in ((B, 1.0), (D, -1.0), (B.T, 1.0), (D.T, -1.0)):
        x = rng.uniform(-1.0, 1.0, n)
        e = x[:h] + x[::-1][:h]
        o = x[:h] - x[::-1][:h]
        E = 0.5 * (A[:h, :h] + A[:h, ::-1][:, :h])
        O = 0.5 * (A[:h, :h] - A[:h, ::-1][:, :h])
        a = E @ e + (A[:h, h] * x[h] if n % 2 else 0.0)
        b = O @ o
        y = np.empty(n)
        y[:h] = a + b
        y[::-1][:h] = sgn * (a - b)
        if n % 2:
            y[h] = A[h, :h] @ (e if sgn > 0 else o) + (A[h, h] * x[h] if sgn > 0 else 0.0)
        assert np.allclose(y, A @ x, atol=1e-12 * np.abs(A).sum(axis=1).max())
