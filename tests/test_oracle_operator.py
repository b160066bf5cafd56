"""Pins of the oracle's SMPM operator (Eq. smpm_poisson, Sec. 1.2-1.4) that do
not depend on the oracle itself: the constant right null vector, rank
deficiency one, exact reproduction of polynomial solutions (with non-zero
Neumann data), spectral convergence on the manufactured cosine problem, and the
split L = A + E B of Sec. 1.3."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.smpm import SMPMGrid, W, E, S, N
from oracle.schur import SchurSystem
from oracle import methods
from paper_1601_03432_gb300 import inputs

TINY = [(2, 2, 6, 1.0, 1.0), (3, 2, 5, 1.0, 1.0), (2, 3, 7, 1.5, 0.75), (4, 3, 4, 2.0, 1.0)]


@pytest.mark.parametrize("mx,my,n,Lx,Ly", TINY)
def test_constant_right_null_and_rank(mx, my, n, Lx, Ly):
    g = SMPMGrid(mx, my, n, Lx, Ly)
    Lm = g.assemble_L()
    one = np.ones(g.r)
    assert np.abs(Lm @ one).max() < 1e-12 * abs(Lm).max()
    s = np.linalg.svd(Lm.toarray(), compute_uv=False)
    assert s[-1] < 1e-12 * s[0]
    assert s[-2] > 1e-7 * s[0]


@pytest.mark.parametrize("mx,my,n,Lx,Ly", TINY)
def test_split_L_equals_A_plus_EB(mx, my, n, Lx, Ly):
    g = SMPMGrid(mx, my, n, Lx, Ly)
    Lm = g.assemble_L()
    A = sp.block_diag([sp.csr_matrix(g.element_A(e)) for e in range(g.nel)], format="csr")
    Em, Bm = g.assemble_E(), g.assemble_B()
    diff = Lm - A - Em @ Bm
    assert abs(diff).max() < 1e-12 * abs(Lm).max()
    # E^T E = I except for the duplicated corner slots (one slot per face node)
    ETE = (Em.T @ Em).toarray()
    assert np.array_equal(np.diag(ETE), np.ones(g.k))
    off = ETE - np.eye(g.k)
    corners = sum(1 for e in range(g.nel) for (F, G) in ((W, S), (W, N), (E, S), (E, N))
                  if g.neighbour(e, F) >= 0 and g.neighbour(e, G) >= 0)
    assert off.sum() == 2 * corners


@pytest.mark.parametrize("mx,my,n,Lx,Ly", TINY)
def test_element_blocks_invertible(mx, my, n, Lx, Ly):
    g = SMPMGrid(mx, my, n, Lx, Ly)
    for e in range(g.nel):
        s = np.linalg.svd(g.element_A(e), compute_uv=False)
        assert s[-1] > 1e-9 * s[0]


@pytest.mark.parametrize("mx,my,n,Lx,Ly", [(2, 2, 5, 1.0, 1.0), (3, 2, 6, 1.5, 0.75), (2, 3, 4, 1.0, 2.0)])
def test_polynomial_solution_is_exact(mx, my, n, Lx, Ly):
    """A cubic u is represented exactly with n >= 4 points, so L u = f + tau g
    must hold to round-off, with g = n.grad u on the physical boundary."""
    g = SMPMGrid(mx, my, n, Lx, Ly)
    x, y = g.coords()
    f, u, gfun = inputs.polynomial_problem(x, y)
    b = g.rhs(f, g.boundary_g(gfun))
    Lm = g.assemble_L()
    res = Lm @ u - b
    assert np.abs(res).max() < 1e-10 * np.abs(b).max()
    # a compatible b is orthogonal to the left null vector
    uL, _ = methods.left_null_L_dense(Lm)
    assert abs(uL @ b) < 1e-10 * np.linalg.norm(b)
    ud = methods.direct_solve(g, Lm, uL, b)
    np.testing.assert_allclose(ud, g.zero_mean(u), atol=1e-9 * np.abs(u).max())


def test_spectral_convergence_in_n():
    """Config-1 problem: the error must fall exponentially with n (Sec. 3.1)."""
    errs = []
    for n in (4, 6, 8, 10, 12):
        g = SMPMGrid(2, 2, n)
        x, y = g.coords()
        f, u = inputs.cos_problem(x, y)
        Lm = g.assemble_L()
        uL, _ = methods.left_null_L_dense(Lm)
        ud = methods.direct_solve(g, Lm, uL, f)
        errs.append(np.abs(ud - g.zero_mean(u)).max())
    errs = np.array(errs)
    assert errs[-1] < 1e-10
    assert np.all(errs[1:] < errs[:-1] * 0.05), errs


def test_algebraic_convergence_in_h():
    """At fixed n the error falls polynomially with h (Sec. 3.1): halving h at
    n = 5 (degree 4) gains a factor between 2^3 and 2^6, i.e. an observed order
    between 3 and 6, not the unbounded gain of p-refinement."""
    errs = []
    for m in (4, 8, 16):
        g = SMPMGrid(m, m, 5)
        x, y = g.coords()
        f, u = inputs.cos_problem(x, y)
        sysm = SchurSystem(g)
        ud = methods.direct_solve(g, g.assemble_L(), sysm.u_L, f)
        errs.append(np.abs(ud - g.zero_mean(u)).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 2 ** 3) and np.all(ratios < 2 ** 6), ratios


@pytest.mark.parametrize("mx,my,n,Lx,Ly", TINY)
def test_element_block_is_mass_symmetric_negative_definite(mx, my, n, Lx, Ly):
    """With tau_F = -n(n-1)/h_perp the collocation face terms equal the GLL
    weak form divided by the nodal mass (integration by parts is exact for the
    degree-(2n-3) integrands), so diag(mass) A_e is symmetric and negative
    definite.  This pins the value and sign of tau and the corner handling."""
    g = SMPMGrid(mx, my, n, Lx, Ly)
    Me = np.outer(g.w1d, g.w1d).ravel()          # w_b w_a at local index b*n + a
    for e in range(g.nel):
        K = Me[:, None] * g.element_A(e)
        assert np.abs(K - K.T).max() < 1e-11 * np.abs(K).max()
        assert np.linalg.eigvalsh(0.5 * (K + K.T)).max() < 0
