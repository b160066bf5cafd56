"""Reverse-mode derivative of the zero-mean solve u(f, g) (test infrastructure).

The forward map of Algorithms 1-3 is linear in (f, g):
    b  = f + tau g                         (Eq. smpm_poisson)
    b~ = Pi b,  Pi = I - u_L u_L^T         (Eq. regularize_poisson)
    L z = b~,   u = N z,  N = I - 1 w^T / (1^T w)   (zero GLL-weighted mean)
For a loss l(u) with gradient gbar = dl/du, put y = N^T gbar = gbar - w (1^T gbar) / (1^T w).
Then 1^T y = 0, so L^T lam = y is consistent (range L^T = 1-perp), and
    <gbar, du> = <y, dz> = <L^T lam, dz> = <lam, Pi db> = <Pi lam, db>,
so dl/db = Pi lam, dl/df = dl/db, and dl/dg on a physical-boundary slot
(e, F, t) is tau_F dl/db at the face node of that slot.

The transposed Schur system (Sec. 1.3 transposed): from L^T = A^T + B^T E^T,
with mu = E^T lam,
    S^T mu = E^T A^-T y,   S^T = I + E^T A^-T B^T,   lam = A^-T (y - B^T mu).
Algorithm 3 runs on S^T with the transposed block-Jacobi blocks M_b^T, the
same interface indicators Z and the coarse matrix C^T = Z^T S^T Z.  The null
vectors swap roles: the left null vector of S^T is the right null vector B 1
of S; the left null vector of C^T is c0 and its right null vector is u_C.
Reading for the singular coarse solve (as in the forward solve, with the
roles swapped): C^T \\ r is the y with C^T y = r - c0^ (c0^T r), u_C^T y = 0,
c0^ = c0 / ||c0||, from the bordered [[C^T, u_C], [u_C^T, 0]].
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .gmres import gmres
from .smpm import W, E, S, N


def zero_mean_transpose(grid, gbar):
    """y = N^T gbar = gbar - w (1^T gbar) / (1^T w), w the GLL mass."""
    w = grid.mass()
    return gbar - w * (gbar.sum() / w.sum())


def grad_f_g(grid, db):
    """dl/df = dl/db; dl/dg per padded slot: tau_F dl/db(face node) on
    physical-boundary faces (b = f + tau g, Eq. smpm_poisson), zero elsewhere."""
    dg = np.zeros(grid.kp)
    for e in range(grid.nel):
        for F in (W, E, S, N):
            if grid.neighbour(e, F) >= 0:
                continue
            for t in range(grid.n):
                a, b = grid.face_node(F, t)
                dg[e * 4 * grid.n + F * grid.n + t] = grid.tau(F, e) * db[grid.node(e, a, b)]
    return db.copy(), dg


def adjoint_direct(grid, Lm, u_L, gbar):
    """dl/db from the plain definition: L^T lam = N^T gbar, solved with the
    nonsingular bordered system [[L^T, 1], [u_L^T, 0]] [lam; eta] = [y; 0]
    (eta = 0 since 1^T y = 0; u_L^T lam = 0 makes lam = Pi lam)."""
    y = zero_mean_transpose(grid, gbar)
    K = sp.bmat([[Lm.T, sp.csr_matrix(np.ones((grid.r, 1)))],
                 [sp.csr_matrix(u_L[None, :]), None]], format="csc")
    sol = spla.splu(K).solve(np.concatenate([y, [0.0]]))
    return sol[: grid.r]


class AdjointDeflation:
    """Coarse objects of the transposed system: C^T, its regularised solve,
    and P', Q' of Eq. projection1/projection2 with S^T in place of S."""

    def __init__(self, sysm):
        self.sysm = sysm
        d = sysm.grid.d
        if not sysm.coarse_singular:   # graded grid: C^T is nonsingular
            self.C_lu = sla.lu_factor(sysm.C.T)
            return
        self.c0hat = sysm.c0 / np.linalg.norm(sysm.c0)
        K = np.zeros((d + 1, d + 1))
        K[:d, :d] = sysm.C.T
        K[:d, d] = sysm.u_C
        K[d, :d] = sysm.u_C
        self.K_lu = sla.lu_factor(K)

    def coarse_solve(self, r):
        if not self.sysm.coarse_singular:
            return sla.lu_solve(self.C_lu, r)
        d = self.sysm.grid.d
        rr = r - self.c0hat * (self.c0hat @ r)
        return sla.lu_solve(self.K_lu, np.concatenate([rr, [0.0]]))[:d]

    def apply_P(self, y):
        s = self.sysm
        return y - s.apply_ST(s.Z @ self.coarse_solve(s.Z.T @ y))

    def apply_Q(self, x):
        s = self.sysm
        return x - s.Z @ self.coarse_solve(s.Z.T @ s.apply_ST(x))


def algorithm3_adjoint(sysm, gbar, tol=1e-10, restart=50, maxit=2000, defl=None):
    """dl/db by Algorithm 3 on the transposed Schur system: right-hand side
    c = E^T A^-T y projected out of B 1 / ||B 1||, mu from the deflated
    block-Jacobi GMRES on S^T, then lam = A^-T (y - B^T mu) and Pi lam."""
    g = sysm.grid
    defl = defl or AdjointDeflation(sysm)
    y = zero_mean_transpose(g, gbar)
    c = sysm.E.T @ sysm.AT_solve(y)
    v = sysm.B1 / np.linalg.norm(sysm.B1)
    c = c - v * (v @ c)
    op = lambda q: defl.apply_P(sysm.apply_ST(sysm.apply_MinvT(q)))
    q, info = gmres(op, defl.apply_P(c), tol, restart, maxit)
    mu = defl.apply_Q(sysm.apply_MinvT(q)) + sysm.Z @ defl.coarse_solve(sysm.Z.T @ c)
    lam = sysm.AT_solve(y - sysm.B.T @ mu)
    db = lam - sysm.u_L * (sysm.u_L @ lam)
    info["schur_relres"] = float(np.linalg.norm(c - sysm.apply_ST(mu)) / max(np.linalg.norm(c), 1e-300))
    return db, info
