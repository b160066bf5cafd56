"""Pins of the oracle's Schur-level objects (Sec. 1.3, 1.4, 2): null vectors,
block-Jacobi blocks, the coarse operator and the deflation projections."""
import numpy as np
import pytest

from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import methods

GRIDS = [(2, 2, 6, 1.0, 1.0), (3, 2, 5, 1.5, 0.75), (3, 3, 4, 1.0, 1.0), (4, 3, 5, 1.0, 2.0)]


@pytest.fixture(scope="module", params=GRIDS, ids=lambda p: "x".join(map(str, p[:3])))
def system(request):
    mx, my, n, Lx, Ly = request.param
    g = SMPMGrid(mx, my, n, Lx, Ly)
    return g, SchurSystem(g)


def test_schur_right_null_is_B1(system):
    g, s = system
    assert np.abs(s.apply_S(s.B1)).max() < 1e-11 * np.abs(s.B1).max()


def test_left_null_vectors(system):
    """u_S (bordered transposed solve) is the dense left singular vector of S,
    and u_S is parallel to E^T u_L with u_L the dense left singular vector of L
    (u_L^T L = 0 and L = A + EB give (E^T u_L)^T S = 0)."""
    g, s = system
    Sd = s.S.toarray()
    U, sv, _ = np.linalg.svd(Sd)
    assert sv[-1] < 1e-11 * sv[0] and sv[-2] > 1e-6 * sv[0]
    assert abs(abs(U[:, -1] @ s.u_S) - 1) < 1e-11
    uL, _ = methods.left_null_L_dense(g.assemble_L())
    assert abs(abs(uL @ s.u_L) - 1) < 1e-11
    v = s.E.T @ uL
    assert abs(abs(v @ s.u_S) / np.linalg.norm(v) - 1) < 1e-11
    assert np.abs(s.u_S @ Sd).max() < 1e-11 * np.abs(Sd).max()


def test_blocks(system):
    """Fig. 2: blocks of 8n (interior), 6n (edge) or 4n (corner) slots that
    partition Gamma; M_b is S restricted to the block."""
    g, s = system
    sizes = sorted(set(len(b) for b in s.blocks))
    assert set(sizes) <= {4 * g.n, 6 * g.n, 8 * g.n, 2 * g.n}
    v = np.random.default_rng(0).standard_normal(g.k)
    Mv = np.zeros(g.k)
    for idx in s.blocks:
        Mv[idx] = s.S[idx][:, idx] @ v[idx]
    np.testing.assert_allclose(s.apply_Minv(Mv), v, rtol=1e-9, atol=1e-9)


def test_SMinv_is_identity_on_white_slots(system):
    """Each white element's slots lie in a black block whose rows of S only
    involve that block, so (S M^-1 v) equals v there (an exact identity)."""
    g, s = system
    v = np.random.default_rng(1).standard_normal(g.k)
    y = s.apply_S(s.apply_Minv(v))
    white = np.array([i for i, (e, F, t) in enumerate(g.slots) if sum(g.element_ij(e)) % 2 == 1])
    np.testing.assert_allclose(y[white], v[white], rtol=1e-10, atol=1e-10)


def test_coarse_operator(system):
    g, s = system
    C = s.C
    assert np.abs(C @ s.c0).max() < 1e-11 * np.abs(C).max()
    sv = np.linalg.svd(C, compute_uv=False)
    assert sv[-1] < 1e-11 * sv[0] and sv[-2] > 1e-8 * sv[0]
    assert np.abs(s.u_C @ C).max() < 1e-11 * np.abs(C).max()
    # C C^+ C = C for the regularised coarse solve
    CCC = np.column_stack([C @ s.coarse_solve(C[:, j]) for j in range(g.d)])
    np.testing.assert_allclose(CCC, C, atol=1e-10 * np.abs(C).max())


def test_projections(system):
    g, s = system
    rng = np.random.default_rng(2)
    y = rng.standard_normal(g.k)
    Py = s.apply_P(y)
    np.testing.assert_allclose(s.apply_P(Py), Py, atol=1e-9 * np.abs(Py).max())
    Qy = s.apply_Q(y)
    np.testing.assert_allclose(s.apply_Q(Qy), Qy, atol=1e-9 * np.abs(Qy).max())
    np.testing.assert_allclose(s.apply_P(s.apply_S(y)), s.apply_S(s.apply_Q(y)), atol=1e-9 * np.abs(y).max())
    Zc = s.Z @ rng.standard_normal(g.d)
    assert np.abs(s.apply_P(s.apply_S(Zc))).max() < 1e-9 * np.abs(Zc).max()
