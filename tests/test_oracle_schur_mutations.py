"""Planted mistakes in the oracle's Schur-level objects and Algorithms 1-3
(Sec. 1.3, 1.4, 2 and Algorithm 3): each plausible error must make at least
one pin fail.  The pins are fixed by the mathematics, not by the oracle's own
formulas: the direct bordered solve of L u = b~ (assembled from the operator,
not from the Schur pieces), dense SVDs of S and L for the null vectors, the
block restriction of the assembled S for M, C C^+ C = C, and the projector
identities P^2 = P, P S = S Q, P S Z = 0.  Some mistakes leave every
algorithm's solution right (a wrong preconditioner or coarse solve only slows
or stops deflating the iteration); the operator pins catch those.  The
mistakes are planted in the oracle, on the CPU."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import methods
from paper_1601_03432_gb300 import inputs


def _close(a, b, rel):
    return np.linalg.norm(a - b) <= rel * max(np.linalg.norm(b), 1e-300)


def first_failing_schur_pin(mx=3, my=2, n=5, Lx=1.5, Ly=0.75):
    """Name of the first pin that fails, or None when all hold."""
    g = SMPMGrid(mx, my, n, Lx, Ly)
    s = SchurSystem(g)
    Sd = s.S.toarray()
    Lm = g.assemble_L()
    # right null vector of S: B 1 (L 1 = 0)
    if np.abs(s.apply_S(s.B1)).max() > 1e-11 * np.abs(s.B1).max():
        return 'S B1 = 0'
    # apply_S is the assembled S
    v = np.random.default_rng(0).standard_normal(g.k)
    if not _close(s.apply_S(v), Sd @ v, 1e-12):
        return 'apply_S = assembled S'
    # left null vectors against dense SVDs of S and L
    U, _, _ = np.linalg.svd(Sd)
    if abs(abs(U[:, -1] @ s.u_S) - 1) > 1e-10:
        return 'u_S = dense SVD'
    UL, _, _ = np.linalg.svd(Lm.toarray())
    if abs(abs(UL[:, -1] @ s.u_L) - 1) > 1e-10:
        return 'u_L = dense SVD'
    # M^-1 inverts S restricted to each block (Fig. 2), colours by i_x + i_y
    Mv = np.zeros(g.k)
    for idx in s.blocks:
        Mv[idx] = Sd[np.ix_(idx, idx)] @ v[idx]
    if not _close(s.apply_Minv(Mv), v, 1e-9):
        return 'M^-1 M_b = I'
    white = np.array([i for i, (e, F, t) in enumerate(g.slots) if (e % mx + e // mx) % 2 == 1])
    if not _close(s.apply_S(s.apply_Minv(v))[white], v[white], 1e-10):
        return 'S M^-1 = I on white slots'
    # C^+ is a generalised inverse of C = Z^T S Z (dense, from the assembled S)
    Zd = s.Z.toarray()
    C = Zd.T @ Sd @ Zd
    CCC = np.column_stack([C @ s.coarse_solve(C[:, j]) for j in range(g.d)])
    if np.abs(CCC - C).max() > 1e-10 * np.abs(C).max():
        return 'C C^+ C = C'
    # projector identities
    y = np.random.default_rng(2).standard_normal(g.k)
    Py = s.apply_P(y)
    if not _close(s.apply_P(Py), Py, 1e-9) or not _close(s.apply_P(Sd @ y), Sd @ s.apply_Q(y), 1e-9):
        return 'P^2 = P, P S = S Q'
    Zc = Zd @ np.random.default_rng(3).standard_normal(g.d)
    if np.abs(s.apply_P(Sd @ Zc)).max() > 1e-9 * np.abs(Sd @ Zc).max():
        return 'P S Z = 0'
    # Algorithms 1-3 against the direct solve, f and Neumann data both non-zero
    b = g.rhs(inputs.white_noise(g.r, 5), np.random.default_rng(6).standard_normal(g.kp))
    ud = methods.direct_solve(g, Lm, s.u_L, b)
    for alg in (methods.algorithm1, methods.algorithm2, methods.algorithm3):
        u, info = alg(s, b, tol=1e-12, maxit=400)
        if not info["converged"] or not _close(u, ud, 1e-9):
            return alg.__name__ + " vs direct solve"
    return None


# ------------------------------------------------------------ the mistakes
def _S_without_identity(self, v):
    return self.B @ self.A_solve(self.E @ v)


def _schur_rhs_sign(self, b):
    return -(self.B @ self.A_solve(b))


def _recover_sign(self, b, x):
    return self.A_solve(b + self.E @ x)


def _Minv_transposed(self, v):
    out = np.zeros_like(v)
    for idx, lu in zip(self.blocks, self.block_lu):
        out[idx] = sla.lu_solve(lu, v[idx], trans=1)
    return out


def _coarse_none(self, r):
    return np.zeros(self.grid.d)


def _P_without_S(self, y):
    return y - self.Z @ self.coarse_solve(self.Z.T @ y)


def _Q_as_P(self, x):
    return x - self.apply_S(self.Z @ self.coarse_solve(self.Z.T @ x))


def _uS_is_right_null(self):
    return self.B1 / np.linalg.norm(self.B1)


def _uL_without_transpose(self):
    y = -self.A_solve(self.B.T @ self.u_S)
    return y / np.linalg.norm(y)


def _no_poisson_projection(sysm, b):
    return b.copy()


def _algorithm3_without_coarse_part(sysm, b, tol=1e-10, restart=50, maxit=2000):
    """Algorithm 3 with the coarse term of Eq. deflated_schur (x2 = Z C^+ Z^T b_S) left out."""
    g = sysm.grid
    b = methods.project_rhs(sysm, b)
    bS = methods.schur_rhs_projected(sysm, b)
    op = lambda v: sysm.apply_P(sysm.apply_S(sysm.apply_Minv(v)))
    x1, info = methods.gmres(op, sysm.apply_P(bS), tol, restart, maxit)
    x = sysm.apply_Q(sysm.apply_Minv(x1))
    return g.zero_mean(sysm.recover(b, x)), info


# Not a mistake, so not planted: leaving out the u_S projection of b_S
# (Eq. regularize_schur).  After b~ = b - u_L u_L^T b, u_L being parallel to
# A^-T B^T u_S gives u_S^T B A^-1 b~ = 0, so that projection only removes
# round-off; every pin above holds without it.
MUTATIONS = [
    (SchurSystem, "apply_S", _S_without_identity),
    (SchurSystem, "schur_rhs", _schur_rhs_sign),
    (SchurSystem, "recover", _recover_sign),
    (SchurSystem, "apply_Minv", _Minv_transposed),
    (SchurSystem, "coarse_solve", _coarse_none),
    (SchurSystem, "apply_P", _P_without_S),
    (SchurSystem, "apply_Q", _Q_as_P),
    (SchurSystem, "left_null_S", _uS_is_right_null),
    (SchurSystem, "left_null_L_from_uS", _uL_without_transpose),
    (methods, "project_rhs", _no_poisson_projection),
    (methods, "algorithm3", _algorithm3_without_coarse_part),
]


def test_unmutated_schur_pins_hold():
    assert first_failing_schur_pin() is None


@pytest.mark.parametrize("target,name,fn", MUTATIONS, ids=[f.__name__.lstrip("_") for _, _, f in MUTATIONS])
def test_planted_schur_mistake_is_caught(monkeypatch, target, name, fn):
    monkeypatch.setattr(target, name, fn)
    try:
        failed = first_failing_schur_pin()
    except Exception as e:      # the oracle's own consistency checks count too
        failed = "exception: %s" % e
    assert failed is not None
