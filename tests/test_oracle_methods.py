"""Pins of Algorithms 1-3 and the GMRES of the oracle: agreement with the
direct bordered solve, manufactured solutions with non-zero Neumann data, and
the paper's qualitative iteration counts (Sec. 3.2, 3.3)."""
import numpy as np
import pytest

from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle.gmres import gmres
from oracle import methods
from paper_1601_03432_gb300 import inputs

ALGS = [methods.algorithm1, methods.algorithm2, methods.algorithm3]


def test_gmres_against_dense_solve():
    rng = np.random.default_rng(3)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, info = gmres(lambda v: A @ v, b, 1e-12, restart=10, maxit=500)
    assert info["converged"]
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10)
    # full GMRES on an n x n system converges in at most n steps
    x, info = gmres(lambda v: A @ v, b, 1e-13, restart=n, maxit=n)
    assert info["iterations"] <= n and info["true_relres"] < 1e-12


def test_gmres_is_the_minimal_residual_method():
    """GMRES's defining property: after j steps from x0 = 0 the residual is
    min over x in K_j(A, b) of ||b - A x||.  Checked step by step against a
    least-squares solve on an orthonormal basis of the Krylov space (a
    different route to the same minimum), plus the properties that follow:
    a non-increasing history, a returned iterate whose true residual is that
    minimum, and termination in 3 steps when A has 3 distinct eigenvalues
    (minimal polynomial of degree 3)."""
    rng = np.random.default_rng(8)
    n = 30
    A = np.eye(n) * 2 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    _, info = gmres(lambda v: A @ v, b, 1e-14, restart=n, maxit=12)
    K = np.empty((n, 12))
    k = b / np.linalg.norm(b)
    for j in range(12):
        K[:, j] = k
        k = A @ k
        k /= np.linalg.norm(k)
    for j in range(1, 13):
        Qj, _ = np.linalg.qr(K[:, :j])
        c, *_ = np.linalg.lstsq(A @ Qj, b, rcond=None)
        rmin = np.linalg.norm(b - A @ (Qj @ c)) / np.linalg.norm(b)
        assert abs(info["history"][j - 1] - rmin) <= 1e-10 + 1e-8 * rmin, (j, info["history"][j - 1], rmin)
    h = info["history"]
    assert all(h[i + 1] <= h[i] * (1 + 1e-12) for i in range(len(h) - 1))
    assert abs(info["true_relres"] - h[-1]) <= 1e-10 + 1e-8 * h[-1]   # the iterate attains the minimum
    # three distinct eigenvalues, non-normal (a random similarity)
    X = rng.standard_normal((n, n)) + np.sqrt(n) * np.eye(n)
    D = np.repeat([1.0, 2.0, 3.5], [10, 10, 10])
    A3 = X @ np.diag(D) @ np.linalg.inv(X)
    x, info = gmres(lambda v: A3 @ v, b, 1e-9, restart=n, maxit=n)
    assert info["converged"] and info["iterations"] <= 3, info["iterations"]
    np.testing.assert_allclose(x, np.linalg.solve(A3, b), rtol=1e-7)


@pytest.mark.parametrize("mx,my,n,Lx,Ly", [(2, 2, 8, 1.0, 1.0), (3, 2, 6, 1.5, 0.75), (4, 4, 5, 1.0, 1.0)])
def test_algorithms_match_direct_solve(mx, my, n, Lx, Ly):
    g = SMPMGrid(mx, my, n, Lx, Ly)
    s = SchurSystem(g)
    x, y = g.coords()
    f = inputs.white_noise(g.r, 5)
    b = g.rhs(f, np.random.default_rng(6).standard_normal(g.kp))
    ud = methods.direct_solve(g, g.assemble_L(), s.u_L, b)
    for alg in ALGS:
        u, info = alg(s, b, tol=1e-12)
        assert info["converged"]
        assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud), alg.__name__


def test_config1_cos_problem():
    g = SMPMGrid(2, 2, 8)
    s = SchurSystem(g)
    x, y = g.coords()
    f, u = inputs.cos_problem(x, y)
    uh, info = methods.algorithm3(s, f, tol=1e-12)
    assert info["converged"] and info["schur_relres"] < 1e-11
    assert np.abs(uh - g.zero_mean(u)).max() < 1e-6


def test_polynomial_with_neumann_data():
    g = SMPMGrid(3, 2, 5, 1.5, 1.0)
    s = SchurSystem(g)
    x, y = g.coords()
    f, u, gfun = inputs.polynomial_problem(x, y)
    b = g.rhs(f, g.boundary_g(gfun))
    uh, info = methods.algorithm3(s, b, tol=1e-13)
    np.testing.assert_allclose(uh, g.zero_mean(u), atol=1e-9 * np.abs(u).max())


def _iters(m, n, alg):
    g = SMPMGrid(m, m, n)
    s = SchurSystem(g)
    x, y = g.coords()
    f, _ = inputs.paper_problem(x, y)
    _, info = alg(s, f, tol=1e-10, restart=300, maxit=600)
    assert info["converged"]
    return info["iterations"]


def test_p_refinement_iterations_flat():
    """Sec. 3.3: with block-Jacobi (and deflation) the count stays nearly flat
    in p at m = 4 (the paper: under 15 preconditioned, under 40 for all)."""
    c3 = [_iters(4, n, methods.algorithm3) for n in (5, 9, 13)]
    c1 = [_iters(4, n, methods.algorithm1) for n in (5, 9, 13)]
    assert max(c3) <= 20 and max(c3) - min(c3) <= 6, c3
    assert max(c1) <= 40, c1


def test_h_refinement_deflation_tempers_growth():
    """Sec. 3.2: the unpreconditioned count grows with m while the deflated
    count stays nearly flat (n = 5)."""
    a1 = [_iters(m, 5, methods.algorithm1) for m in (4, 8, 16)]
    a3 = [_iters(m, 5, methods.algorithm3) for m in (4, 8, 16)]
    assert a1[2] > 2 * a1[0], a1
    assert max(a3) <= 20 and a3[2] < a1[2] / 2, (a1, a3)
