"""Planted mistakes: each plausible error in the oracle's operator must make at
least one of its pins fail.  The mistakes are planted in the oracle, on the CPU."""
import numpy as np
import pytest

import oracle.smpm as sm
from oracle.smpm import SMPMGrid
from paper_1601_03432_gb300 import inputs


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


def _swap_h(self, F, t):
    n = self.n
    row = np.zeros(self.nn)
    sx, sy = 2.0 / self.hy, 2.0 / self.hx           # mistake: h_x and h_y swapped
    if F == sm.W:
        row[t * n + np.arange(n)] = -sx * self.D[0]
    elif F == sm.E:
        row[t * n + np.arange(n)] = sx * self.D[n - 1]
    elif F == sm.S:
        row[np.arange(n) * n + t] = -sy * self.D[0]
    else:
        row[np.arange(n) * n + t] = sy * self.D[n - 1]
    return row


def _neighbour_sign(self, F, t):
    G = sm.OPPOSITE[F]
    row = self.normal_derivative_row(G, t)          # mistake: neighbour normal not negated
    a, b = self.face_node(G, t)
    row[b * self.n + a] += self.robin_weight(F)
    return row


def _neighbour_reversed(self, F, t):
    G = sm.OPPOSITE[F]
    t2 = self.n - 1 - t                             # mistake: face nodes matched in reverse
    row = -self.normal_derivative_row(G, t2)
    a, b = self.face_node(G, t2)
    row[b * self.n + a] += self.robin_weight(F)
    return row


def _tau_sign(self, F):
    h = self.hx if F in (sm.W, sm.E) else self.hy
    return self.tau_scale * self.n * (self.n - 1) / h  # mistake: wrong sign


def _tau_scale2(self, F):
    h = self.hx if F in (sm.W, sm.E) else self.hy
    return -2.0 * self.n * (self.n - 1) / h          # mistake: factor 2


def _laplacian_dropped(self):
    I = np.eye(self.n)
    D2 = self.D @ self.D
    return (2.0 / self.hx) ** 2 * np.kron(I, D2)     # mistake: y term dropped


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
