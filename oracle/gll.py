"""Gauss-Lobatto-Legendre nodes, weights and differentiation matrix.

Sec. 1.2: each element carries an n x n GLL grid; derivatives are taken with
spectral differentiation matrices (the paper cites Costa & Don 2000 for them and
for their round-off behaviour).  With N = n - 1 the nodes are -1, +1 and the
roots of P_N', the weights are 2 / (N (N+1) P_N(x_j)^2), and the
differentiation matrix is the derivative of the Lagrange interpolant,
D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)) for i != j, with the diagonal taken as
minus the off-diagonal row sum (the round-off remedy of Costa & Don).
"""
import numpy as np


def legendre(N, x):
    """P_N(x), P_N'(x) and P_N''(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p_prev, p = np.ones_like(x), x.copy()
    dp_prev, dp = np.zeros_like(x), np.ones_like(x)
    if N == 0:
        return p_prev, dp_prev, np.zeros_like(x)
    for k in range(1, N):
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        dp_next = dp_prev + (2 * k + 1) * p
        p_prev, p = p, p_next
        dp_prev, dp = dp, dp_next
    # Legendre's equation (1 - x^2) P'' - 2 x P' + N(N+1) P = 0 gives P''
    # away from x = +-1 (only used at interior Newton iterates).
    with np.errstate(divide="ignore", invalid="ignore"):
        ddp = (2 * x * dp - N * (N + 1) * p) / (1 - x * x)
    return p, dp, ddp


def gll_nodes_weights(n):
    """n GLL nodes on [-1, 1] (increasing) and their quadrature weights."""
    if n < 2:
        raise ValueError("need n >= 2 GLL points")
    N = n - 1
    # interior nodes: roots of P_N', Newton from Chebyshev-Gauss-Lobatto guesses
    xi = -np.cos(np.pi * np.arange(1, N) / N)
    for _ in range(100):
        _, dp, ddp = legendre(N, xi)
        step = dp / ddp
        xi = xi - step
        if np.all(np.abs(step) < 1e-16):
            break
    x = np.concatenate([[-1.0], xi, [1.0]])
    pN, _, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * pN ** 2)
    return x, w


def diff_matrix(x):
    """Spectral differentiation matrix on the GLL nodes x (Sec. 1.2)."""
    n = len(x)
    N = n - 1
    pN, _, _ = legendre(N, x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = pN[i] / (pN[j] * (x[i] - x[j]))
    for i in range(n):
        D[i, i] = -sum(D[i, j] for j in range(n) if j != i)
    return D
