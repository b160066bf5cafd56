"""Pins of the oracle's adjoint (reverse-mode derivative of u(f, g)).

Each pin uses only the forward direct solve (the plain definition of u) and
the mathematics of a linear map: brute-force transposition of the forward
map on tiny grids, the inner-product identity, and central finite
differences of a quadratic loss."""
import numpy as np
import pytest

from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import methods, adjoint
from paper_1601_03432_gb300 import inputs

GRIDS = [(2, 2, 5, 1.0, 1.0), (3, 2, 5, 1.5, 0.75), (3, 3, 4, 1.0, 1.0)]


def _setup(mx, my, n, Lx, Ly):
    g = SMPMGrid(mx, my, n, Lx, Ly)
    s = SchurSystem(g)
    return g, s, g.assemble_L()


def _forward_matrix(g, s, Lm):
    """Columns u(e_i) of the forward map b -> u, by the direct solve."""
    G = np.empty((g.r, g.r))
    for i in range(g.r):
        b = np.zeros(g.r)
        b[i] = 1.0
        G[:, i] = methods.direct_solve(g, Lm, s.u_L, b)
    return G


@pytest.mark.parametrize("mx,my,n,Lx,Ly", GRIDS)
def test_direct_adjoint_is_transpose_of_forward_map(mx, my, n, Lx, Ly):
    g, s, Lm = _setup(mx, my, n, Lx, Ly)
    G = _forward_matrix(g, s, Lm)
    gbar = np.random.default_rng(1).standard_normal(g.r) + 0.3   # non-zero sum
    db = adjoint.adjoint_direct(g, Lm, s.u_L, gbar)
    np.testing.assert_allclose(db, G.T @ gbar, atol=1e-10 * np.abs(db).max())


@pytest.mark.parametrize("mx,my,n,Lx,Ly", GRIDS)
def test_algorithm3_adjoint_matches_direct(mx, my, n, Lx, Ly):
    g, s, Lm = _setup(mx, my, n, Lx, Ly)
    gbar = inputs.white_noise(g.r, 9) + 0.5
    db_ref = adjoint.adjoint_direct(g, Lm, s.u_L, gbar)
    db, info = adjoint.algorithm3_adjoint(s, gbar, tol=1e-12)
    assert info["converged"]
    assert np.linalg.norm(db - db_ref) <= 1e-9 * np.linalg.norm(db_ref)


def test_inner_product_identity_with_algorithm3():
    g, s, Lm = _setup(4, 3, 6, 1.0, 1.0)
    rng = np.random.default_rng(4)
    gbar = rng.standard_normal(g.r)
    db, _ = adjoint.algorithm3_adjoint(s, gbar, tol=1e-13)
    for k in range(3):
        dbv = rng.standard_normal(g.r)
        u, _ = methods.algorithm3(s, dbv, tol=1e-13)
        lhs, rhs = gbar @ u, db @ dbv
        assert abs(lhs - rhs) <= 1e-9 * (np.linalg.norm(gbar) * np.linalg.norm(u))


def test_grad_f_g_by_central_differences():
    """loss = ||u - u_t||^2 is quadratic and u is linear in (f, g), so
    central differences carry no truncation error; h = 1e-3 keeps rounding
    small against the direct solve."""
    g, s, Lm = _setup(3, 2, 5, 1.0, 1.0)
    rng = np.random.default_rng(11)
    x, y = g.coords()
    f, _ = inputs.fourier_rhs(x, y, seed=5)
    gg = rng.standard_normal(g.kp)
    ut = rng.standard_normal(g.r)

    def loss(ff, gv):
        u = methods.direct_solve(g, Lm, s.u_L, g.rhs(ff, gv))
        return float(((u - ut) ** 2).sum()), u

    l0, u0 = loss(f, gg)
    db = adjoint.adjoint_direct(g, Lm, s.u_L, 2 * (u0 - ut))
    df, dg = adjoint.grad_f_g(g, db)
    h = 1e-3
    for k in range(6):
        pf = rng.standard_normal(g.r)
        pg = rng.standard_normal(g.kp)
        fd = (loss(f + h * pf, gg + h * pg)[0] - loss(f - h * pf, gg - h * pg)[0]) / (2 * h)
        an = df @ pf + dg @ pg
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1.0)
    # only physical-boundary slots carry a g-derivative
    for e in range(g.nel):
        for F in range(4):
            sl = slice(e * 4 * g.n + F * g.n, e * 4 * g.n + (F + 1) * g.n)
            if g.neighbour(e, F) >= 0:
                assert np.all(dg[sl] == 0.0)


def test_adjoint_coarse_solve_is_generalised_inverse():
    g, s, _ = _setup(4, 4, 5, 1.0, 1.0)
    defl = adjoint.AdjointDeflation(s)
    rng = np.random.default_rng(2)
    z = rng.standard_normal(g.d)
    Ct = s.C.T
    y = defl.coarse_solve(Ct @ z)
    np.testing.assert_allclose(Ct @ y, Ct @ z, atol=1e-10 * np.abs(Ct @ z).max())
    assert abs(s.u_C @ y) < 1e-12 * np.linalg.norm(y)
    # c0 is the left null vector of C^T
    assert np.abs(s.c0 @ Ct).max() < 1e-10 * np.abs(Ct).max() * np.linalg.norm(s.c0)


# ------------------------------------------------------- planted mistakes
def _adjoint_pins_hold():
    """The brute-force transpose pin on Algorithm 3's adjoint and the
    central-difference pin on the g-derivative, on one small grid."""
    g, s, Lm = _setup(3, 2, 4, 1.5, 0.75)
    G = _forward_matrix(g, s, Lm)
    gbar = np.random.default_rng(1).standard_normal(g.r) + 0.3
    db, _ = adjoint.algorithm3_adjoint(s, gbar, tol=1e-12)
    if np.linalg.norm(db - G.T @ gbar) > 1e-8 * np.linalg.norm(db):
        return False
    rng = np.random.default_rng(3)
    gg = rng.standard_normal(g.kp)
    f = np.zeros(g.r)
    df, dg = adjoint.grad_f_g(g, db)
    pg = rng.standard_normal(g.kp)
    h = 1e-3
    up = methods.direct_solve(g, Lm, s.u_L, g.rhs(f, gg + h * pg))
    um = methods.direct_solve(g, Lm, s.u_L, g.rhs(f, gg - h * pg))
    fd = gbar @ (up - um) / (2 * h)
    return abs(fd - dg @ pg) <= 1e-7 * max(abs(fd), 1.0)


def _no_zero_mean_transpose(grid, gbar):
    return gbar.copy()                                   # mistake: N^T dropped


def _grad_sign(grid, db):
    df, dg = _ORIG_GRAD(grid, db)
    return df, -dg                                       # mistake: sign of tau


def _no_transpose_solve(self, b):
    return self.A_solve(b)                               # mistake: A^-1 for A^-T


_ORIG_GRAD = adjoint.grad_f_g


def test_unmutated_adjoint_pins_hold():
    assert _adjoint_pins_hold()


@pytest.mark.parametrize("target,name,fn", [
    (adjoint, "zero_mean_transpose", _no_zero_mean_transpose),
    (adjoint, "grad_f_g", _grad_sign),
    (SchurSystem, "AT_solve", _no_transpose_solve),
])
def test_planted_adjoint_mistake_is_caught(monkeypatch, target, name, fn):
    monkeypatch.setattr(target, name, fn)
    assert not _adjoint_pins_hold()
