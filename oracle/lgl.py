"""Legendre-Gauss-Lobatto collocation (Sec. 2.2.1, "Domain decomposition":
N LGL points per dimension on the reference interval) and the Lagrange basis
of Eqs. (field_expansion) and (lagrprod), evaluated directly from its product
formula.

Test infrastructure: slow, plain FP64, imported only by tests and by the
CPU-baseline leg of the benchmark.
"""
import numpy as np


def legendre(n, x):
    """P_n(x) and P_n'(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=float)
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0, np.zeros_like(x)
    for m in range(1, n):
        p0, p1 = p1, ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
    # derivative from (1 - x^2) P_n' = n (P_{n-1} - x P_n), away from x = +-1
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (p0 - x * p1) / (1.0 - x * x)
    end = np.isclose(np.abs(x), 1.0)
    dp = np.where(end, np.sign(x) ** (n + 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def lgl_nodes_weights(N):
    """N LGL nodes (ascending) and weights: the end points -1, +1 and the
    roots of P'_{N-1}; weights 2 / (N (N-1) P_{N-1}(x)^2)."""
    if N < 2:
        raise ValueError("LGL needs N >= 2")
    n = N - 1
    x = -np.cos(np.pi * np.arange(N) / n)  # Chebyshev-Lobatto start
    for _ in range(100):
        P, dP = legendre(n, x[1:-1])
        # Legendre ODE: (1 - x^2) P'' = 2 x P' - n (n + 1) P
        d2P = (2 * x[1:-1] * dP - n * (n + 1) * P) / (1.0 - x[1:-1] ** 2)
        step = dP / d2P
        x[1:-1] -= step
        if np.max(np.abs(step), initial=0.0) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    P, _ = legendre(n, x)
    w = 2.0 / (N * n * P ** 2)
    return x, w


def lagrange(nodes, j, x):
    """l_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m)."""
    out = np.ones_like(np.asarray(x, dtype=float))
    for m, xm in enumerate(nodes):
        if m != j:
            out = out * (x - xm) / (nodes[j] - xm)
    return out


def lagrange_deriv(nodes, j, x):
    """l_j'(x) = sum_{k != j} 1/(x_j - x_k) prod_{m != j,k} (x - x_m)/(x_j - x_m)."""
    x = np.asarray(x, dtype=float)
    out = np.zeros_like(x)
    for k, xk in enumerate(nodes):
        if k == j:
            continue
        term = np.full_like(x, 1.0 / (nodes[j] - xk))
        for m, xm in enumerate(nodes):
            if m != j and m != k:
                term = term * (x - xm) / (nodes[j] - xm)
        out = out + term
    return out


def diff_matrix(nodes):
    """D[i, j] = l_j'(x_i): derivative at node i of the interpolant of nodal data."""
    N = len(nodes)
    D = np.zeros((N, N))
    for j in range(N):
        D[:, j] = lagrange_deriv(nodes, j, nodes)
    return D


def interp_matrix(nodes, x):
    """I[q, j] = l_j(x_q)."""
    x = np.asarray(x, dtype=float)
    return np.stack([lagrange(nodes, j, x) for j in range(len(nodes))], axis=1)
