"""Pins of the oracle's GLL nodes, weights and differentiation matrix (Sec. 1.2)
against closed forms, exact quadrature and the node list drawn in Fig. 1."""
import os

import numpy as np
import pytest

from oracle.gll import gll_nodes_weights, diff_matrix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_gll_n11.txt")


def test_closed_form_small_n():
    x, w = gll_nodes_weights(3)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-14)
    x, w = gll_nodes_weights(4)
    s = 1 / np.sqrt(5)
    np.testing.assert_allclose(x, [-1, -s, s, 1], rtol=1e-14)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-14)
    x, w = gll_nodes_weights(5)
    s = np.sqrt(3 / 7)
    np.testing.assert_allclose(x, [-1, -s, 0, s, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=1e-14)


def test_fig1_node_list():
    drawn = np.loadtxt(GOLDEN)
    x, _ = gll_nodes_weights(11)
    assert np.all(np.abs(x - drawn) <= 0.005 + 1e-12)


@pytest.mark.parametrize("n", range(2, 31))
def test_weights_and_quadrature(n):
    x, w = gll_nodes_weights(n)
    assert np.all(np.diff(x) > 0)
    np.testing.assert_allclose(w.sum(), 2.0, rtol=1e-14)
    # GLL quadrature with n points integrates polynomials of degree <= 2n - 3 exactly
    for m in range(0, 2 * n - 2):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(w @ x ** m - exact) < 1e-13
    # the bound is sharp: for P_N^2 (degree 2N) the GLL rule gives 2/N instead
    # of the exact 2/(2N+1) (a classical closed form)
    if n > 2:
        from numpy.polynomial import legendre as npleg
        c = np.zeros(n)
        c[-1] = 1.0
        pN = npleg.legval(x, c)
        np.testing.assert_allclose(w @ pN ** 2, 2.0 / (n - 1), rtol=1e-12)


@pytest.mark.parametrize("n", range(2, 31))
def test_differentiation_matrix(n):
    x, _ = gll_nodes_weights(n)
    D = diff_matrix(x)
    N = n - 1
    for m in range(0, N + 1):
        exact = m * x ** (m - 1) if m > 0 else np.zeros(n)
        err = np.abs(D @ x ** m - exact).max()
        assert err < 1e-13 * n ** 2 * max(1, m)
    # closed-form diagonal: -N(N+1)/4, 0 (interior), +N(N+1)/4
    np.testing.assert_allclose(D[0, 0], -N * (N + 1) / 4, rtol=1e-12)
    np.testing.assert_allclose(D[-1, -1], N * (N + 1) / 4, rtol=1e-12)
    if n > 2:
        assert np.abs(np.diag(D)[1:-1]).max() < 1e-11 * n ** 2
