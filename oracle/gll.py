"""Gauss-Lobatto-Legendre (GLL) tables for the oracle.  TEST INFRASTRUCTURE ONLY.

Sec. 3.2 of arXiv:1806.01422 represents the solution on each element by the
nodal Lagrange basis through the N+1 GLL points of [-1, 1] (Legendre polynomials
on a GLL grid, chosen over Chebyshev for milder time-step limits).  The mass
matrix is diagonal (the GLL quadrature weights) and the "differential matrix"
reduces to the quadrature weights times the collocation derivative because the
basis functions are one at their own node and zero at the others.

This module writes out the textbook definitions:

* nodes: x_0 = -1, x_N = +1 and the N-1 roots of P_N'(x);
* weights: w_i = 2 / (N (N+1) P_N(x_i)^2);
* collocation derivative D_ij = l_j'(x_i) in the closed form
  D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)) for i != j,
  D_00 = -N(N+1)/4, D_NN = +N(N+1)/4, other diagonal entries 0.
"""
import numpy as np


def legendre(N, x):
    """P_N(x) and P_{N-1}(x) by the three-term recurrence (k+1)P_{k+1} = (2k+1)xP_k - kP_{k-1}."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if N == 0:
        return p_prev, np.zeros_like(x)
    p = x.copy()
    for k in range(1, N):
        p_prev, p = p, ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
    return p, p_prev


def gll_nodes_weights(N):
    """N+1 GLL nodes (ascending) and weights on [-1, 1] (Sec. 3.2).

    Interior nodes are the roots of P_N'; they are found by Newton's method on
    q(x) = (1 - x^2) P_N'(x), started from the Chebyshev-Gauss-Lobatto points.
    With (1 - x^2) P_N' = N (P_{N-1} - x P_N), Newton's step needs q and q' =
    -N (N+1) P_N (Legendre's equation).
    """
    if N < 1:
        raise ValueError("GLL needs order N >= 1")
    x = -np.cos(np.pi * np.arange(N + 1) / N)
    inner = x[1:-1].copy()
    for _ in range(100):
        pN, pN1 = legendre(N, inner)
        q = N * (pN1 - inner * pN)
        dq = -N * (N + 1) * pN
        step = q / dq
        inner -= step
        if np.max(np.abs(step), initial=0.0) < 1e-16:
            break
    x[1:-1] = inner
    x[0], x[-1] = -1.0, 1.0
    pN, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * pN ** 2)
    return x, w


def derivative_matrix(N, x):
    """Collocation derivative D_ij = l_j'(x_i) on the GLL nodes (closed form, Sec. 3.2)."""
    n = N + 1
    pN, _ = legendre(N, x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = pN[i] / (pN[j] * (x[i] - x[j]))
    D[0, 0] = -N * (N + 1) / 4.0
    D[N, N] = N * (N + 1) / 4.0
    return D


def gll(N):
    """(nodes, weights, derivative matrix) for order N."""
    x, w = gll_nodes_weights(N)
    return x, w, derivative_matrix(N, x)
