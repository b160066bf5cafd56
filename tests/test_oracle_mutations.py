"""Planted mistakes: each plausible error in the oracle's operator must make at
least one of its pins fail.  The mistakes are planted in the oracle, on the CPU.

The identity weight p_F of the Robin flux is invisible to the operator
identities (L 1 = 0, polynomial exactness and mass symmetry hold for any p_F),
so its mistakes are checked against the entry-by-entry pins: the hand-derived
n = 2 operators and the polynomial derivation of L."""
import os

import numpy as np
import pytest

import oracle.smpm as sm
from oracle.smpm import SMPMGrid
from paper_1601_03432_gb300 import inputs
from smpm_by_polynomials import operator_by_polynomials, read_golden_n2, golden_matrix


def pins_hold(mx=3, my=2, n=5, Lx=1.5, Ly=0.75):
    g = SMPMGrid(mx, my, n, Lx, Ly)
    Lm = g.assemble_L()
    x, y = g.coords()
    f, u, gfun = inputs.polynomial_problem(x, y)
    b = g.rhs(f, g.boundary_g(gfun))
    if np.abs(Lm @ u - b).max() > 1e-10 * np.abs(b).max():
        return False
    if np.abs(Lm @ np.ones(g.r)).max() > 1e-12 * abs(Lm).max():
        return False
    Me = np.outer(g.w1d, g.w1d).ravel()
    for e in range(g.nel):
        K = Me[:, None] * g.element_A(e)
        if np.abs(K - K.T).max() > 1e-11 * np.abs(K).max():
            return False
        if np.linalg.eigvalsh(0.5 * (K + K.T)).max() >= 0:
            return False
    return True


def _swap_h(self, F, t, e):
    n = self.n
    row = np.zeros(self.nn)
    hx, hy = self.h_of(e)
    sx, sy = 2.0 / hy, 2.0 / hx                     # mistake: h_x and h_y swapped
    if F == sm.W:
        row[t * n + np.arange(n)] = -sx * self.D[0]
    elif F == sm.E:
        row[t * n + np.arange(n)] = sx * self.D[n - 1]
    elif F == sm.S:
        row[np.arange(n) * n + t] = -sy * self.D[0]
    else:
        row[np.arange(n) * n + t] = sy * self.D[n - 1]
    return row


def _neighbour_sign(self, F, t, e):
    G = sm.OPPOSITE[F]
    row = self.normal_derivative_row(G, t, self.neighbour(e, F))  # mistake: neighbour normal not negated
    a, b = self.face_node(G, t)
    row[b * self.n + a] += self.robin_weight(F, e)
    return row


def _neighbour_reversed(self, F, t, e):
    G = sm.OPPOSITE[F]
    t2 = self.n - 1 - t                             # mistake: face nodes matched in reverse
    row = -self.normal_derivative_row(G, t2, self.neighbour(e, F))
    a, b = self.face_node(G, t2)
    row[b * self.n + a] += self.robin_weight(F, e)
    return row


def _tau_sign(self, F, e):
    return self.tau_scale * self.n * (self.n - 1) / self.h_perp(F, e)  # mistake: wrong sign


def _tau_scale2(self, F, e):
    return -2.0 * self.n * (self.n - 1) / self.h_perp(F, e)          # mistake: factor 2


def _laplacian_dropped(self, e):
    I = np.eye(self.n)
    D2 = self.D @ self.D
    return (2.0 / self.h_of(e)[0]) ** 2 * np.kron(I, D2)     # mistake: y term dropped


def _face_node_swapped(self, F, t):
    n = self.n
    return {sm.W: (t, 0), sm.E: (t, n - 1), sm.S: (0, t), sm.N: (n - 1, t)}[F]  # W/E vs S/N mixed


MUTATIONS = [
    ("normal_derivative_row", _swap_h),
    ("neighbour_robin_row", _neighbour_sign),
    ("neighbour_robin_row", _neighbour_reversed),
    ("tau", _tau_sign),
    ("tau", _tau_scale2),
    ("laplacian_block", _laplacian_dropped),
    ("face_node", _face_node_swapped),
]


def test_unmutated_pins_hold():
    assert pins_hold()


@pytest.mark.parametrize("name,fn", MUTATIONS, ids=[f.__name__ for _, f in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, fn):
    monkeypatch.setattr(sm.SMPMGrid, name, fn)
    try:
        ok = pins_hold()
    except Exception:
        ok = False
    assert not ok


# ---- the Robin identity weight p_F -------------------------------------------
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "L_n2_two_element_grids.txt")


def robin_pins_hold():
    gold = read_golden_n2(GOLDEN)
    for grid, (mx, my) in (("2x1", (2, 1)), ("1x2", (1, 2))):
        for literal in (False, True):
            hx, hy = 3.0 / mx, 2.0 / my
            px, py = (1.0, 1.0) if literal else (0.5 / hx, 0.5 / hy)
            Lg = golden_matrix(gold[grid], hx, hy, px, py)
            Lo = SMPMGrid(mx, my, 2, 3.0, 2.0, robin_literal=literal).assemble_L().toarray()
            if np.abs(Lo - Lg).max() > 1e-13 * np.abs(Lg).max():
                return False
    for mx, my, n in ((2, 2, 3), (2, 3, 4)):
        Lp = operator_by_polynomials(mx, my, n, 1.5, 0.6)
        Lo = SMPMGrid(mx, my, n, 1.5, 0.6).assemble_L().toarray()
        if np.abs(Lo - Lp).max() > 1e-11 * np.abs(Lp).max():
            return False
    return True


def _robin_h_swapped(self, F, e):
    if self.robin_literal:
        return 1.0
    hx, hy = self.h_of(e)
    h = hy if F in (sm.W, sm.E) else hx               # mistake: h_perp taken along the face
    return self.robin_scale * self.n * (self.n - 1) / h


def _robin_hx_everywhere(self, F, e):
    if self.robin_literal:
        return 1.0
    return self.robin_scale * self.n * (self.n - 1) / self.h_of(e)[0]   # mistake: h_x on S/N faces too


def _robin_no_quarter(self, F, e):
    if self.robin_literal:
        return 1.0
    return self.n * (self.n - 1) / self.h_perp(F, e)  # mistake: the factor 1/4 dropped


def _robin_master_gradient(self, F, e):
    if self.robin_literal:
        return 1.0
    return 2.0 / self.h_perp(F, e)                    # mistake: 2/h (master-element scale) for n(n-1)/(4h)


def _robin_literal_ignored(self, F, e):
    return self.robin_scale * self.n * (self.n - 1) / self.h_perp(F, e)   # mistake: the literal reading not honoured


def _robin_identity_on_own_side_only(self, F, t, e):
    G = sm.OPPOSITE[F]
    return -self.normal_derivative_row(G, t, self.neighbour(e, F))  # mistake: neighbour's p_F u' term dropped


ROBIN_MUTATIONS = [
    ("robin_weight", _robin_h_swapped),
    ("robin_weight", _robin_hx_everywhere),
    ("robin_weight", _robin_no_quarter),
    ("robin_weight", _robin_master_gradient),
    ("robin_weight", _robin_literal_ignored),
    ("neighbour_robin_row", _robin_identity_on_own_side_only),
]


def test_unmutated_robin_pins_hold():
    assert robin_pins_hold()


@pytest.mark.parametrize("name,fn", ROBIN_MUTATIONS, ids=[f.__name__ for _, f in ROBIN_MUTATIONS])
def test_planted_robin_mistake_is_caught(monkeypatch, name, fn):
    monkeypatch.setattr(sm.SMPMGrid, name, fn)
    try:
        ok = robin_pins_hold()
    except Exception:
        ok = False
    assert not ok


@pytest.mark.parametrize("fn", [_robin_h_swapped, _robin_no_quarter], ids=["h_swapped", "no_quarter"])
def test_robin_mistakes_pass_the_operator_identities(monkeypatch, fn):
    """Why the entry-by-entry pins are needed: these weight mistakes keep
    L 1 = 0, polynomial exactness and mass symmetry."""
    monkeypatch.setattr(sm.SMPMGrid, "robin_weight", fn)
    assert pins_hold()
