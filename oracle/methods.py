"""Algorithms 1, 2 and 3 of the paper and the direct reference solve.

Every algorithm takes the discrete right-hand side b = f + tau g
(Eq. smpm_poisson) and returns the zero-mean u together with solver info.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .gmres import gmres


def project_rhs(sysm, b):
    """Projection of the right-hand side out of the left null space of L
    (Eq. regularize_poisson, Sec. 1.4): b <- b - u_L u_L^T b."""
    return b - sysm.u_L * (sysm.u_L @ b)


def schur_rhs_projected(sysm, b):
    """Schur right-hand side of Eq. schur_complement_system, b_S = B A^-1 b,
    projected out of the left null space of S (Eq. regularize_schur):
    b_S <- b_S - u_S (u_S^T b_S)."""
    bS = sysm.schur_rhs(b)
    return bS - sysm.u_S * (sysm.u_S @ bS)


def algorithm1(sysm, b, tol=1e-10, restart=50, maxit=2000):
    """Algorithm 1 (Sec. 1.4): GMRES on the regularised Schur system
    S x_S = b_S (Eqs. schur_complement_system, regularize_schur), then
    u = A^-1 (b - E x_S) and the zero-mean normalisation."""
    g = sysm.grid
    b = project_rhs(sysm, b)
    bS = schur_rhs_projected(sysm, b)
    xS, info = gmres(sysm.apply_S, bS, tol, restart, maxit)
    u = sysm.recover(b, xS)
    return g.zero_mean(u), info


def algorithm2(sysm, b, tol=1e-10, restart=50, maxit=2000):
    """Algorithm 2: right block-Jacobi preconditioned Schur method,
    x' = GMRES(S M^-1, b_S), x = M^-1 x' (Sec. 2)."""
    g = sysm.grid
    b = project_rhs(sysm, b)
    bS = schur_rhs_projected(sysm, b)
    xp, info = gmres(lambda v: sysm.apply_S(sysm.apply_Minv(v)), bS, tol, restart, maxit)
    x = sysm.apply_Minv(xp)
    u = sysm.recover(b, x)
    return g.zero_mean(u), info


def algorithm3(sysm, b, tol=1e-10, restart=50, maxit=2000):
    """Algorithm 3: deflated and block-Jacobi preconditioned Schur method,
    Eq. (deflated_schur):
        x_S = Z C\\(Z^T - u_C u_C^T Z^T) b_S + Q M^-1 GMRES(P S M^-1, P b_S)."""
    g = sysm.grid
    b = project_rhs(sysm, b)
    bS = schur_rhs_projected(sysm, b)
    # the deflated, right-preconditioned system P S M^-1 y = P b_S and the two
    # terms of Eq. deflated_schur
    op = lambda v: sysm.apply_P(sysm.apply_S(sysm.apply_Minv(v)))
    y, info = gmres(op, sysm.apply_P(bS), tol, restart, maxit)
    x1 = sysm.apply_Q(sysm.apply_Minv(y))
    x2 = sysm.Z @ sysm.coarse_solve(sysm.Z.T @ bS)
    x = x1 + x2
    u = sysm.recover(b, x)
    info["schur_relres"] = float(np.linalg.norm(bS - sysm.apply_S(x)) / max(np.linalg.norm(bS), 1e-300))
    return g.zero_mean(u), info


def direct_solve(grid, Lm, u_L, b):
    """Reference solution of the regularised system L u = b~ (Eq.
    regularize_poisson), b~ = b - u_L u_L^T b, normalised to zero GLL mean by
    the nonsingular bordered system [[L, 1], [w^T, 0]] [u; mu] = [b~; 0] with w
    the GLL mass (mu = 0 because b~ is in the range of L)."""
    bt = b - u_L * (u_L @ b)
    w = grid.mass()
    K = sp.bmat([[Lm, sp.csr_matrix(np.ones((grid.r, 1)))],
                 [sp.csr_matrix(w[None, :]), None]], format="csc")
    sol = spla.splu(K).solve(np.concatenate([bt, [0.0]]))
    return sol[: grid.r]


def left_null_L_dense(Lm):
    """Unit left singular vector of L for its smallest singular value (dense
    SVD; small grids only), sign fixed by the largest-magnitude entry."""
    U, s, Vt = np.linalg.svd(Lm.toarray())
    v = U[:, -1]
    i = int(np.argmax(np.abs(v)))
    return (v if v[i] >= 0 else -v), s
