"""Pins of the oracle's Robin flux R = p_F I + n.grad and penalty tau_F
(Eq. smpm_poisson, Sec. 1.2) that every operator identity misses: L 1 = 0,
rank r - 1, L = A + E B, polynomial exactness and mass symmetry hold for any
identity weight p_F, so the weight is pinned entry by entry.

* The n = 2 operators of a 2x1 and a 1x2 grid on a rectangle (L_x != L_y,
  so h_x != h_y on both), derived by hand (tests/golden/L_n2_two_element_grids.txt,
  derivation in its header), under both readings of the weight.
* L for n = 2..5 on several grids, computed from Lagrange polynomials in
  physical coordinates (tests/smpm_by_polynomials.py), for the scaled reading
  p_F = beta n(n-1)/h_perp (beta = 1/4 and another beta), the literal reading
  p_F = 1, and a non-default penalty scale.
"""
import os

import numpy as np
import pytest

from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import methods
from paper_1601_03432_gb300 import inputs
from smpm_by_polynomials import operator_by_polynomials, read_golden_n2, golden_matrix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "L_n2_two_element_grids.txt")
LX, LY = 3.0, 2.0


@pytest.mark.parametrize("grid", ["2x1", "1x2"])
@pytest.mark.parametrize("literal", [False, True])
def test_n2_operator_matches_hand_derivation(grid, literal):
    mx, my = (2, 1) if grid == "2x1" else (1, 2)
    g = SMPMGrid(mx, my, 2, LX, LY, robin_literal=literal)
    hx, hy = LX / mx, LY / my
    px, py = (1.0, 1.0) if literal else (0.5 / hx, 0.5 / hy)   # n(n-1)/(4h) = 1/(2h) at n = 2
    Lg = golden_matrix(read_golden_n2(GOLDEN)[grid], hx, hy, px, py)
    assert np.allclose(Lg.sum(axis=1), 0.0, atol=1e-14)           # the derivation itself: L 1 = 0
    Lo = g.assemble_L().toarray()
    assert np.abs(Lo - Lg).max() <= 1e-13 * np.abs(Lg).max(), np.abs(Lo - Lg).max()


CASES = [
    (2, 1, 3), (1, 2, 3), (2, 2, 3), (3, 2, 4), (2, 3, 5), (2, 2, 2), (1, 3, 4),
]


@pytest.mark.parametrize("mx,my,n", CASES)
@pytest.mark.parametrize("reading", ["scaled", "scaled_beta", "literal", "tau"])
def test_operator_matches_polynomial_derivation(mx, my, n, reading):
    Lx, Ly = 1.5, 0.6
    kw = {"scaled": {}, "scaled_beta": {"robin_scale": 0.7}, "literal": {"robin_literal": True},
          "tau": {"tau_scale": 1.3}}[reading]
    g = SMPMGrid(mx, my, n, Lx, Ly, **kw)
    Lp = operator_by_polynomials(mx, my, n, Lx, Ly, tau_scale=kw.get("tau_scale", 1.0),
                                 robin_scale=kw.get("robin_scale", 0.25), literal=kw.get("robin_literal", False))
    Lo = g.assemble_L().toarray()
    assert np.abs(Lo - Lp).max() <= 1e-11 * np.abs(Lp).max(), np.abs(Lo - Lp).max()


def test_literal_reading_solves_match_direct_solve():
    """The solver identities hold under the literal weight too: Algorithms 1-3
    agree with the bordered direct solve of L (Sec. 1.3 - 2)."""
    g = SMPMGrid(3, 2, 6, 1.5, 0.75, robin_literal=True)
    s = SchurSystem(g)
    f = inputs.white_noise(g.r, 5)
    b = g.rhs(f, np.random.default_rng(6).standard_normal(g.kp))
    ud = methods.direct_solve(g, g.assemble_L(), s.u_L, b)
    for alg in (methods.algorithm1, methods.algorithm2, methods.algorithm3):
        u, info = alg(s, b, tol=1e-12)
        assert info["converged"]
        assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud), alg.__name__
