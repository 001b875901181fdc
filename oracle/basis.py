"""1D ingredients of the tensor-product Q_p basis (oracle; test infrastructure only).

Sec. 2.3: nodal basis on Legendre-Gauss-Lobatto (LGL/GLL) points, Gauss quadrature.
Fig. 1 prints the p=4 LGL points on [0,1] as 0, .1727, .5, .8273, 1.

All points live on the reference interval [0,1].
"""
from __future__ import annotations

import numpy as np


def legendre_and_derivative(n: int, x: np.ndarray):
    """P_n(x) and P_n'(x) by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},  P'_{k+1} = P'_{k-1} + (2k+1) P_k."""
    x = np.asarray(x, dtype=np.float64)
    p_prev, p = np.ones_like(x), x.copy()
    dp_prev, dp = np.zeros_like(x), np.ones_like(x)
    if n == 0:
        return p_prev, dp_prev
    for k in range(1, n):
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        dp_next = dp_prev + (2 * k + 1) * p
        p_prev, p = p, p_next
        dp_prev, dp = dp, dp_next
    return p, dp


def gll_nodes(p: int) -> np.ndarray:
    """The p+1 Gauss-Lobatto-Legendre points on [0,1]: the end points plus the
    roots of P_p' (Newton's method on P_p', with P_p'' from Legendre's ODE
    (1-x^2) P'' = 2x P' - p(p+1) P)."""
    if p < 1:
        raise ValueError("order must be >= 1")
    if p == 1:
        return np.array([0.0, 1.0])
    x = -np.cos(np.pi * np.arange(1, p) / p)          # interior initial guesses on [-1,1]
    for _ in range(100):
        P, dP = legendre_and_derivative(p, x)
        d2P = (2 * x * dP - p * (p + 1) * P) / (1 - x * x)
        step = dP / d2P
        x = x - step
        if np.max(np.abs(step)) < 1e-16:
            break
    x = np.concatenate(([-1.0], x, [1.0]))
    x = 0.5 * (x - x[::-1])                            # exact symmetry about 0
    return 0.5 * (x + 1.0)


def gauss_rule(q: int):
    """q-point Gauss-Legendre rule on [0,1]: points are the roots of P_q (Newton),
    weights 2 / ((1 - x^2) P_q'(x)^2) on [-1,1], halved for [0,1]."""
    if q < 1:
        raise ValueError("q must be >= 1")
    x = -np.cos(np.pi * (np.arange(q) + 0.75) / (q + 0.5))
    for _ in range(100):
        P, dP = legendre_and_derivative(q, x)
        step = P / dP
        x = x - step
        if np.max(np.abs(step)) < 1e-16:
            break
    _, dP = legendre_and_derivative(q, x)
    w = 2.0 / ((1.0 - x * x) * dP * dP)
    x = 0.5 * (x - x[::-1])
    w = 0.5 * (w + w[::-1])
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L[i, j] = l_j(x_i) with l_j(x) = prod_{m != j} (x - r_m) / (r_j - r_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_derivatives(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dL[i, j] = l_j'(x_i) = sum_{m != j} 1/(r_j - r_m) prod_{k != j, m} (x - r_k)/(r_j - r_k)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    dL = np.zeros((len(x), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[m]))
            for k in range(n):
                if k != j and k != m:
                    term *= (x - nodes[k]) / (nodes[j] - nodes[k])
            dL[:, j] += term
    return dL
