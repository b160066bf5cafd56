"""Seeded synthetic inputs for the SMPM Poisson-Neumann solve.

This module draws random numbers and evaluates closed-form fields at points the
caller supplies.  It holds none of the solver's arithmetic (no GLL nodes, no
differentiation, no operators): both the CUDA path and the oracle take their
node coordinates from their own discretisation and pass them in.

Workloads (the paper measures on no public dataset; these stand in for it):

* ``cos_problem``: f = -2 pi^2 cos(pi x) cos(pi y), g = 0 on [0,1]^2 - the
  manufactured problem whose exact solution is cos(pi x) cos(pi y).
* ``paper_problem``: f = cos(lam pi x / L_x) cos(lam pi y / L_y), homogeneous
  Neumann, lam = 7 (the test problem of Sec. 3).
* ``fourier_rhs``: 32 distinct cosine modes (k_x, k_y) in {0..8}^2 \\ {(0,0)}
  with amplitudes N(0,1)/(k_x^2 + k_y^2), numpy PCG64 seeded; every mode has
  zero mean and zero normal derivative on the unit square, so f is compatible
  with g = 0.
* ``white_noise``: i.i.d. N(0,1) nodal values (Sec. 3.3 mentions white-noise
  right-hand sides).
* ``uneven_batch``: a list of (m_x, m_y, n, nrhs) drawn uniformly from
  m in {4..32}, n in {8..24}, nrhs in {1..16}.
* ``polynomial_problem``: u = a cubic polynomial with f = lap u and
  g = n . grad u, whose discrete solution is exact whenever n >= 4.
* ``clustered_edges`` / ``jittered_edges``: element edges of graded grids -
  tanh clustering toward both walls (the element-size profile of
  wall-resolved grids), or uniform edges moved by a seeded fraction of h.
"""
import numpy as np


def cos_problem(x, y):
    """Config-1 problem on [0,1]^2: returns f and the exact u."""
    u = np.cos(np.pi * x) * np.cos(np.pi * y)
    return -2.0 * np.pi ** 2 * u, u


def paper_problem(x, y, lam=7, Lx=1.0, Ly=1.0):
    """Sec. 3 test problem: returns f and the exact zero-mean u."""
    c = np.cos(lam * np.pi * x / Lx) * np.cos(lam * np.pi * y / Ly)
    u = -c / (lam ** 2 * np.pi ** 2 * (1.0 / Lx ** 2 + 1.0 / Ly ** 2))
    return c, u


def fourier_modes(seed, nmodes=32, kmax=8):
    """The seeded list of (k_x, k_y, amplitude)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = [(kx, ky) for kx in range(kmax + 1) for ky in range(kmax + 1) if (kx, ky) != (0, 0)]
    pick = rng.choice(len(pairs), size=nmodes, replace=False)
    amps = rng.standard_normal(nmodes)
    out = []
    for i, p in enumerate(pick):
        kx, ky = pairs[p]
        out.append((kx, ky, amps[i] / (kx * kx + ky * ky)))
    return out


def fourier_rhs(x, y, seed, nmodes=32, kmax=8):
    """Seeded Fourier right-hand side on [0,1]^2: returns f and the exact u."""
    f = np.zeros_like(np.asarray(x, dtype=np.float64))
    u = np.zeros_like(f)
    for kx, ky, a in fourier_modes(seed, nmodes, kmax):
        c = np.cos(kx * np.pi * x) * np.cos(ky * np.pi * y)
        f += a * c
        u -= a * c / (np.pi ** 2 * (kx * kx + ky * ky))
    return f, u


def white_noise(r, seed):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(r)


def uneven_batch(count=512, seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    mx = rng.integers(4, 33, count)
    my = rng.integers(4, 33, count)
    n = rng.integers(8, 25, count)
    nrhs = rng.integers(1, 17, count)
    return [tuple(int(v) for v in t) for t in zip(mx, my, n, nrhs)]


def polynomial_problem(x, y, coeffs=(0.3, -1.1, 0.7, 0.45, -0.2, 0.9)):
    """u = c0 x^3 + c1 x^2 y + c2 x y^2 + c3 y^3 + c4 x y + c5 x^2.
    Returns f = lap u, u, and a function g(x, y, nx, ny) = n . grad u."""
    c0, c1, c2, c3, c4, c5 = coeffs
    u = c0 * x ** 3 + c1 * x ** 2 * y + c2 * x * y ** 2 + c3 * y ** 3 + c4 * x * y + c5 * x ** 2
    f = (6 * c0 * x + 2 * c1 * y + 2 * c5) + (2 * c2 * x + 6 * c3 * y)

    def g(xx, yy, nx, ny):
        ux = 3 * c0 * xx ** 2 + 2 * c1 * xx * yy + c2 * yy ** 2 + c4 * yy + 2 * c5 * xx
        uy = c1 * xx ** 2 + 2 * c2 * xx * yy + 3 * c3 * yy ** 2 + c4 * xx
        return nx * ux + ny * uy

    return f, u, g


def clustered_edges(m, L=1.0, stretch=2.0):
    """m + 1 edges on [0, L] clustered toward both ends by tanh stretching
    (larger stretch, thinner wall elements)."""
    s = np.linspace(-1.0, 1.0, m + 1)
    e = np.tanh(stretch * s) / np.tanh(stretch)
    e = L * (e + 1.0) / 2.0
    e[0], e[-1] = 0.0, L
    return e


def jittered_edges(m, L, seed, amp=0.3):
    """m + 1 edges on [0, L]: interior uniform edges moved by U(-amp, amp) h."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = L / m
    e = np.arange(m + 1) * h
    e[1:-1] += rng.uniform(-amp, amp, m - 1) * h
    return e
