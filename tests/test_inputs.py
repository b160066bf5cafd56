"""The seeded synthetic workloads follow their stated recipe: 32 distinct
cosine modes (k_x, k_y) in {0..8}^2 without (0, 0), amplitudes N(0,1) over
k_x^2 + k_y^2, and an exact solution u with lap u = f, homogeneous Neumann
data and zero mean; the uneven batch draws m_x, m_y in 4..32, n in 8..24 and
1..16 right-hand sides per problem.  Everything is reproducible from the
seed."""
import numpy as np

from paper_1601_03432_gb300 import inputs


def test_fourier_modes_recipe():
    for seed in (1000, 1001, 5, 6):
        modes = inputs.fourier_modes(seed)
        assert len(modes) == 32
        ks = [(kx, ky) for kx, ky, _ in modes]
        assert len(set(ks)) == 32
        assert all(0 <= kx <= 8 and 0 <= ky <= 8 and (kx, ky) != (0, 0) for kx, ky in ks)
        assert modes == inputs.fourier_modes(seed)                      # deterministic
    assert inputs.fourier_modes(1000) != inputs.fourier_modes(1001)
    # amplitudes are N(0,1) draws scaled by 1/(k_x^2 + k_y^2)
    raw = np.concatenate([[a * (kx * kx + ky * ky) for kx, ky, a in inputs.fourier_modes(s)] for s in range(200)])
    assert abs(raw.mean()) < 0.05 and abs(raw.std() - 1.0) < 0.05


def test_fourier_rhs_solution_is_exact():
    """lap u = f by second differences (error O(h^2)), zero normal derivative
    on the boundary and zero mean of f and u over the unit square."""
    h = 1.0 / 400
    t = np.linspace(0.0, 1.0, 401)
    X, Y = np.meshgrid(t, t, indexing="ij")
    f, u = inputs.fourier_rhs(X, Y, seed=1000)
    lap = (u[2:, 1:-1] + u[:-2, 1:-1] + u[1:-1, 2:] + u[1:-1, :-2] - 4 * u[1:-1, 1:-1]) / h ** 2
    assert np.abs(lap - f[1:-1, 1:-1]).max() < 2e-3 * np.abs(f).max()
    for edge in (u[0, :] - u[1, :], u[-1, :] - u[-2, :], u[:, 0] - u[:, 1], u[:, -1] - u[:, -2]):
        assert np.abs(edge).max() < 5e-4 * np.abs(u).max()              # O(h^2) one-sided difference
    w = np.full(401, h)
    w[[0, -1]] = h / 2                                                  # trapezoid weights
    W = np.outer(w, w)
    assert abs((W * f).sum()) < 1e-10 * np.abs(f).max()
    assert abs((W * u).sum()) < 1e-10 * np.abs(u).max()


def test_uneven_batch_recipe():
    probs = inputs.uneven_batch(512, seed=7)
    assert len(probs) == 512 and probs == inputs.uneven_batch(512, seed=7)
    a = np.array(probs)
    assert a[:, :2].min() == 4 and a[:, :2].max() == 32
    assert a[:, 2].min() == 8 and a[:, 2].max() == 24
    assert a[:, 3].min() == 1 and a[:, 3].max() == 16
    assert a[:, 3].sum() == 4460                                        # the benchmark's right-hand-side count
    assert inputs.uneven_batch(512, seed=8) != probs


def test_graded_edges_recipe():
    """Clustered edges: symmetric, strictly increasing, exact end points,
    thinnest at the walls; jittered edges: seeded, within 0.3 h of uniform."""
    for m, L, st in ((8, 1.0, 2.0), (24, 1.3, 2.0), (5, 0.5, 1.5)):
        e = inputs.clustered_edges(m, L, st)
        h = np.diff(e)
        assert e[0] == 0.0 and e[-1] == L and np.all(h > 0)
        np.testing.assert_allclose(e + e[::-1], L, atol=1e-14)      # symmetric about L / 2
        assert h[0] <= h.min() * (1 + 1e-12) and h[len(h) // 2] >= h.max() * (1 - 1e-12)
    assert np.diff(inputs.clustered_edges(24, 1.0, 2.0)).max() / np.diff(inputs.clustered_edges(24, 1.0, 2.0)).min() > 10
    e1, e2 = inputs.jittered_edges(7, 1.4, 3), inputs.jittered_edges(7, 1.4, 3)
    assert np.array_equal(e1, e2) and not np.array_equal(e1, inputs.jittered_edges(7, 1.4, 4))
    u = np.arange(8) * (1.4 / 7)
    assert e1[0] == 0.0 and abs(e1[-1] - 1.4) < 1e-15 and np.all(np.diff(e1) > 0)
    assert np.abs(e1 - u).max() <= 0.3 * 1.4 / 7 + 1e-15
