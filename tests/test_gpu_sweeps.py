"""The paper's refinement studies through the GPU path (Sec. 3.2, 3.3): the
lambda = 7 cosine problem with homogeneous Neumann data on the unit square,
relative tolerance 1e-10, Algorithms 1, 2 and 3 (precond 0, 1, 2), under
h-refinement (m_x = m_y = 4 ... 32 at n = 5) and p-refinement (n = 5 ... 15
at m = 4), and the white-noise right-hand side the paper mentions for the
p-study.  Each GPU iteration count must be within one of the oracle's on the
same problem, and the counts must show the paper's trends: the deflated
count grows much more slowly in h than the unpreconditioned one, and on the
cosine problem the preconditioned counts stay nearly flat in p."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1601_03432_gb300 import Grid, inputs
from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import methods

ALGS = [methods.algorithm1, methods.algorithm2, methods.algorithm3]
RESTART = 200


@pytest.fixture(scope="module")
def built():
    from paper_1601_03432_gb300.build import build
    build()
    assert torch.cuda.is_available()


def gpu_iters(m, n, precond, f):
    lg = Grid(m, m, n)
    lg.factor(tol=1e-10, restart=RESTART, precond=precond)
    u = torch.zeros(lg.r, dtype=torch.float64, device="cuda")
    rep = lg.solve(torch.as_tensor(f, device="cuda"), u)[0]
    lg.close()
    assert rep["converged"] == 1
    return rep["iterations"]


def oracle_iters(m, n, precond, f):
    g = SMPMGrid(m, m, n)
    s = SchurSystem(g)
    _, info = ALGS[precond](s, f, tol=1e-10, restart=RESTART, maxit=2000)
    assert info["converged"]
    return info["iterations"]


@pytest.mark.slow
def test_h_refinement(built):
    table = {}
    for m in (4, 8, 16, 32):
        x, y = SMPMGrid(m, m, 5).coords()
        f, _ = inputs.paper_problem(x, y)
        for p in (0, 1, 2):
            gi, oi = gpu_iters(m, 5, p, f), oracle_iters(m, 5, p, f)
            assert abs(gi - oi) <= 1, (m, p, gi, oi)
            table[m, p] = gi
    # Sec. 3.2: "nearly 110" unpreconditioned at m = 32; deflation tempers the growth
    assert 100 <= table[32, 0] <= 120, table
    assert table[32, 2] < table[32, 0] / 3 and table[32, 2] - table[4, 2] < 10, table


@pytest.mark.slow
@pytest.mark.parametrize("rhs", ["cosine", "white_noise"])
def test_p_refinement(built, rhs):
    table = {}
    for n in (5, 7, 9, 11, 13, 15):
        og = SMPMGrid(4, 4, n)
        x, y = og.coords()
        f = inputs.paper_problem(x, y)[0] if rhs == "cosine" else inputs.white_noise(og.r, 77)
        for p in (0, 1, 2):
            gi, oi = gpu_iters(4, n, p, f), oracle_iters(4, n, p, f)
            assert abs(gi - oi) <= 1, (n, p, gi, oi)
            table[n, p] = gi
    if rhs == "cosine":
        # Sec. 3.3: about 40 at most for every variant (the paper: "less than
        # 40"; 40 here for Algorithm 1 at n = 15), preconditioned counts nearly
        # flat in p (the paper: "under 15"; 12-18 here)
        assert max(table.values()) <= 40, table
        pre = [table[n, p] for n in (5, 7, 9, 11, 13, 15) for p in (1, 2)]
        assert max(pre) <= 20 and max(pre) - min(pre) <= 8, table
    else:
        # a nodal white-noise right-hand side carries the highest modes of
        # every n: the counts grow with p under this reading (Algorithm 3
        # 16 -> 26, Algorithm 1 31 -> 94 for n = 5 -> 15), the deflated
        # and preconditioned ones far less than the plain Schur iteration
        assert all(table[n, 2] < table[n, 0] / 2 for n in (9, 11, 13, 15)), table
