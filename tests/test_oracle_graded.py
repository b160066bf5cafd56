"""Pins of the oracle on graded grids (Sec. 1.2: elements are any smooth
invertible maps of the master square; here axis-aligned rectangles whose
width varies by column and height by row).

On a graded grid every element's factors differ, tau_F and p_F differ across
an interface, and B 1 (the right null vector of S) is no longer constant on
each interface.  With the 0/1 deflation vectors of Sec. 2 the coarse matrix
C = Z^T S Z then becomes nonsingular and B 1 leaves the coarse space; the
oracle's graded reading weights z_j by B 1 (divided by the mean of the two
sides), which keeps B 1 = Z c0 and is the indicator on a uniform grid.  The
pins:

* L computed a second way, from Lagrange polynomials in physical coordinates
  (tests/smpm_by_polynomials.py), entry by entry;
* L 1 = 0 and rank r - 1 (the Neumann problem keeps its one-dimensional null
  space); a global cubic is reproduced exactly; the discrete solution of a
  smooth problem converges spectrally in n;
* diag(mass) A_e symmetric negative definite for every element (the penalty of
  each face uses the element's own size);
* GLL mass: total = area, exact integral of a quartic;
* a grid given by uniform edges is the uniform grid, with singular C;
* Algorithms 1-3 and the adjoint reach the direct solution; with indicator
  vectors C is singular exactly when every interface has the same size across
  it, with weighted vectors always (C c0 = 0, weights 1 on uniform grids);
* on a wall-clustered grid the weighted deflation keeps the iteration count
  near the uniform grid's, while the indicator vectors stagnate.

Planted graded mistakes (the neighbour's gradient taken with the receiving
element's size, the neighbour's own p_F on its trace, the penalty from the
neighbour's size, node coordinates from the mean size) must each fail a pin.
"""
import numpy as np
import pytest

import oracle.smpm as sm
from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import methods, adjoint
from paper_1601_03432_gb300 import inputs
from smpm_by_polynomials import operator_by_polynomials

XS = [0.0, 0.2, 0.5, 1.0, 1.3]
YS = [0.0, 0.35, 0.5, 1.1]


def graded(n, xs=XS, ys=YS, **kw):
    return SMPMGrid(len(xs) - 1, len(ys) - 1, n, xs=xs, ys=ys, **kw)


GRADED_CASES = [
    ([0.0, 0.3, 1.0], [0.0, 1.0], 3),
    ([0.0, 1.0], [0.0, 0.25, 1.2], 4),
    ([0.0, 0.2, 0.5, 1.1], [0.0, 0.6, 0.75], 5),
    ([-0.4, 0.1, 0.3], [1.0, 1.2, 1.7, 1.9], 4),
]


def pins_hold_graded():
    for xs, ys, n in GRADED_CASES[:3]:
        g = SMPMGrid(len(xs) - 1, len(ys) - 1, n, xs=xs, ys=ys)
        Lp = operator_by_polynomials(g.mx, g.my, n, 0, 0, xs=xs, ys=ys)
        if np.abs(g.assemble_L().toarray() - Lp).max() > 1e-11 * np.abs(Lp).max():
            return False
    g = graded(5)
    Lm = g.assemble_L()
    x, y = g.coords()
    f, u, gfun = inputs.polynomial_problem(x, y)
    b = g.rhs(f, g.boundary_g(gfun))
    if np.abs(Lm @ u - b).max() > 1e-10 * np.abs(b).max():
        return False
    Me = np.outer(g.w1d, g.w1d).ravel()
    for e in range(g.nel):
        K = Me[:, None] * g.element_A(e)
        if np.abs(K - K.T).max() > 1e-11 * np.abs(K).max():
            return False
    return True


@pytest.mark.parametrize("xs,ys,n", GRADED_CASES)
@pytest.mark.parametrize("reading", ["scaled", "literal", "tau"])
def test_graded_operator_matches_polynomial_derivation(xs, ys, n, reading):
    kw = {"scaled": {}, "literal": {"robin_literal": True}, "tau": {"tau_scale": 1.3, "robin_scale": 0.6}}[reading]
    g = SMPMGrid(len(xs) - 1, len(ys) - 1, n, xs=xs, ys=ys, **kw)
    Lp = operator_by_polynomials(g.mx, g.my, n, 0, 0, tau_scale=kw.get("tau_scale", 1.0),
                                 robin_scale=kw.get("robin_scale", 0.25), literal=kw.get("robin_literal", False),
                                 xs=xs, ys=ys)
    Lo = g.assemble_L().toarray()
    assert np.abs(Lo - Lp).max() <= 1e-11 * np.abs(Lp).max(), np.abs(Lo - Lp).max()


def test_graded_null_space_and_polynomial_exactness():
    g = graded(5)
    Lm = g.assemble_L()
    assert np.abs(Lm @ np.ones(g.r)).max() < 1e-12 * abs(Lm).max()
    s = np.linalg.svd(Lm.toarray(), compute_uv=False)
    assert s[-1] < 1e-12 * s[0] and s[-2] > 1e-8 * s[0]
    x, y = g.coords()
    f, u, gfun = inputs.polynomial_problem(x, y)
    b = g.rhs(f, g.boundary_g(gfun))
    assert np.abs(Lm @ u - b).max() < 1e-10 * np.abs(b).max()


def test_graded_element_blocks_mass_symmetric_negative_definite():
    g = graded(6)
    Me = np.outer(g.w1d, g.w1d).ravel()
    for e in range(g.nel):
        K = Me[:, None] * g.element_A(e)
        assert np.abs(K - K.T).max() < 1e-11 * np.abs(K).max()
        assert np.linalg.eigvalsh(0.5 * (K + K.T)).max() < 0


def test_graded_mass_and_coordinates():
    g = graded(5)
    x, y = g.coords()
    w = g.mass()
    assert abs(w.sum() - 1.3 * 1.1) < 1e-13
    # GLL quadrature with n = 5 is exact to degree 7 per direction
    exact = (1.3 ** 5 / 5) * (1.1 ** 3 / 3)
    assert abs(w @ (x ** 4 * y ** 2) - exact) < 1e-12 * exact
    assert x.min() == 0.0 and abs(x.max() - 1.3) < 1e-15 and abs(y.max() - 1.1) < 1e-15


def test_graded_spectral_convergence():
    errs = []
    for n in (4, 6, 8, 10):
        g = SMPMGrid(3, 2, n, xs=[0.0, 0.25, 0.45, 1.0], ys=[0.0, 0.7, 1.0])
        x, y = g.coords()
        f, u = inputs.cos_problem(x, y)
        sysm = SchurSystem(g)
        ud = methods.direct_solve(g, g.assemble_L(), sysm.u_L, f)
        errs.append(np.abs(ud - g.zero_mean(u)).max())
    errs = np.array(errs)
    assert errs[-1] < 1e-7 and np.all(errs[1:] < errs[:-1] * 0.1), errs


def test_uniform_edges_give_the_uniform_grid():
    gu = SMPMGrid(4, 3, 5, 1.3, 1.1)
    gg = SMPMGrid(4, 3, 5, xs=np.arange(5) * (1.3 / 4), ys=np.arange(4) * (1.1 / 3))
    A, B = gu.assemble_L(), gg.assemble_L()
    assert abs(A - B).max() < 1e-12 * abs(A).max()
    assert SchurSystem(gg).coarse_singular and SchurSystem(gu).coarse_singular


@pytest.mark.parametrize("xs,ys,singular", [
    ([0.0, 0.5, 1.0, 1.5], [0.0, 0.3, 0.6], True),        # uniform
    ([0.0, 0.5, 1.0, 1.6], [0.0, 0.3, 0.6], False),       # one column wider
    ([0.0, 0.5, 1.0, 1.5], [0.0, 0.3, 0.7], False),       # one row taller
    ([0.0, 0.5, 1.0, 1.5], [0.0, 0.3, 0.6, 1.1], False),  # the last row taller
])
def test_weighted_coarse_space_holds_B1(xs, ys, singular):
    g = SMPMGrid(len(xs) - 1, len(ys) - 1, 4, xs=xs, ys=ys)
    sysm = SchurSystem(g)
    assert sysm.coarse_singular
    assert np.abs(sysm.Z @ sysm.c0 - sysm.B1).max() < 1e-13 * np.abs(sysm.B1).max()
    assert np.abs(sysm.C @ sysm.c0).max() < 1e-10 * np.abs(sysm.C).max() * np.linalg.norm(sysm.c0)
    if singular:   # uniform: exactly the 0/1 vectors of Sec. 2
        assert np.all(sysm.zweights == 1.0)
    else:          # each side's weight is its B 1 over the interface mean
        assert np.abs(sysm.zweights - 1.0).max() > 1e-3
        assert np.allclose(sysm.Z.T @ sysm.Z @ np.ones(g.d) / (2 * g.n), 1.0, atol=0.5)


@pytest.mark.parametrize("xs,ys,singular", [
    ([0.0, 0.5, 1.0, 1.5], [0.0, 0.3, 0.6], True),        # uniform
    ([0.0, 0.5, 1.0, 1.6], [0.0, 0.3, 0.6], False),       # one column wider
    ([0.0, 0.5, 1.0, 1.5], [0.0, 0.3, 0.7], False),       # one row taller
    ([0.0, 0.5, 1.0, 1.5], [0.0, 0.3, 0.6, 1.1], False),  # the last row taller
])
def test_indicator_coarse_matrix_singular_only_when_sizes_match(xs, ys, singular):
    g = SMPMGrid(len(xs) - 1, len(ys) - 1, 4, xs=xs, ys=ys)
    sysm = SchurSystem(g, deflation="indicator")
    assert sysm.coarse_singular == singular
    sv = np.linalg.svd(sysm.C, compute_uv=False)
    if singular:
        assert sv[-1] < 1e-10 * sv[0]
    else:
        assert sv[-1] > 1e-4 * sv[0]
        # S is still singular with the right null vector B 1
        assert np.linalg.norm(sysm.apply_S(sysm.B1)) < 1e-10 * np.linalg.norm(sysm.B1)


@pytest.mark.parametrize("alg,deflation", [("algorithm1", "weighted"), ("algorithm2", "weighted"),
                                           ("algorithm3", "weighted"), ("algorithm3", "indicator")])
def test_graded_algorithms_reach_direct_solution(alg, deflation):
    g = graded(6)
    sysm = SchurSystem(g, deflation=deflation)
    x, y = g.coords()
    f, _ = inputs.fourier_rhs(x, y, seed=5)
    gb = g.boundary_g(lambda X, Y, nx, ny: np.cos(X) * nx + np.sin(Y) * ny)
    b = g.rhs(f, gb)
    ud = methods.direct_solve(g, g.assemble_L(), sysm.u_L, b)
    u, info = getattr(methods, alg)(sysm, b, tol=1e-12)
    assert info["converged"]
    assert np.linalg.norm(u - ud) < 1e-10 * np.linalg.norm(ud)
    if alg == "algorithm3":
        # either coarse space: the two terms of Eq. deflated_schur give
        # S x_S = b_S (the assembly is exact for any coarse solve used
        # consistently in P, Q and the coarse term)
        assert info["schur_relres"] < 1e-10


def test_weighted_deflation_on_wall_clustered_grid():
    """12 x 12 elements, n = 6, tanh-clustered toward the walls (sizes spanning
    a factor of about 10): the weighted coarse space keeps Algorithm 3 well
    below Algorithm 2; the 0/1 vectors leave B 1 outside it and stall."""
    xs = inputs.clustered_edges(12, 1.0, 2.0)
    g = SMPMGrid(12, 12, 6, xs=list(xs), ys=list(xs))
    x, y = g.coords()
    f, _ = inputs.fourier_rhs(x, y, seed=1002)
    b = g.rhs(f)
    its = {}
    for defl in ("weighted", "indicator"):
        sysm = SchurSystem(g, deflation=defl)
        _, info = methods.algorithm3(sysm, b, tol=1e-10, maxit=300)
        its[defl] = info["iterations"] if info["converged"] else 10 ** 6
    _, info2 = methods.algorithm2(sysm, b, tol=1e-10, maxit=300)
    assert its["weighted"] <= 45 and info2["iterations"] > 2 * its["weighted"], (its, info2["iterations"])
    assert its["indicator"] > 4 * its["weighted"], its


def test_graded_adjoint_matches_direct():
    g = graded(5)
    sysm = SchurSystem(g)
    gbar = inputs.white_noise(g.r, 9)
    ref = adjoint.adjoint_direct(g, g.assemble_L(), sysm.u_L, gbar)
    db, info = adjoint.algorithm3_adjoint(sysm, gbar, tol=1e-12)
    assert info["converged"]
    assert np.linalg.norm(db - ref) < 1e-9 * np.linalg.norm(ref)


# ---- planted graded mistakes -------------------------------------------------
def _neighbour_gradient_own_size(self, F, t, e):
    G = sm.OPPOSITE[F]
    row = -self.normal_derivative_row(G, t, e)        # mistake: neighbour's gradient with e's size
    a, b = self.face_node(G, t)
    row[b * self.n + a] += self.robin_weight(F, e)
    return row


def _neighbour_own_weight(self, F, t, e):
    G = sm.OPPOSITE[F]
    e2 = self.neighbour(e, F)
    row = -self.normal_derivative_row(G, t, e2)
    a, b = self.face_node(G, t)
    row[b * self.n + a] += self.robin_weight(G, e2)   # mistake: the neighbour's own p on its trace
    return row


def _tau_from_neighbour(self, F, e):
    e2 = self.neighbour(e, F)
    h = self.h_perp(F, e2 if e2 >= 0 else e)           # mistake: penalty from the neighbour's size
    return -self.tau_scale * self.n * (self.n - 1) / h


def _mean_size(self, e):
    return self.Lx / self.mx, self.Ly / self.my        # mistake: uniform sizes on a graded grid


GRADED_MUTATIONS = [
    ("neighbour_robin_row", _neighbour_gradient_own_size),
    ("neighbour_robin_row", _neighbour_own_weight),
    ("tau", _tau_from_neighbour),
    ("h_of", _mean_size),
]


def test_unmutated_graded_pins_hold():
    assert pins_hold_graded()


@pytest.mark.parametrize("name,fn", GRADED_MUTATIONS, ids=[f.__name__ for _, f in GRADED_MUTATIONS])
def test_planted_graded_mistake_is_caught(monkeypatch, name, fn):
    monkeypatch.setattr(sm.SMPMGrid, name, fn)
    try:
        ok = pins_hold_graded()
    except Exception:
        ok = False
    assert not ok
