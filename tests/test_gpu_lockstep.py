"""Lockstep solves of several right-hand sides (schur_solve with nrhs > 1,
FP64, block-Jacobi with and without deflation): every column against the
oracle's direct bordered solve and its Algorithm 2 / 3 on the same
right-hand side (iteration counts within one), and against the one-at-a-time
solve of the library.  Column counts that are not powers of two, resident
and global operator layouts, a zero right-hand side among others, and
columns that stop at maxit are covered."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1601_03432_gb300 import Grid, inputs
from paper_1601_03432_gb300 import _binding as B
from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import methods


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def built():
    from paper_1601_03432_gb300.build import build
    build()
    assert torch.cuda.is_available()


GRIDS = [(3, 2, 5, 1.5, 0.75), (5, 4, 7, 1.0, 1.0), (9, 7, 5, 1.0, 1.0), (16, 16, 8, 1.0, 1.0)]


@pytest.fixture(scope="module", params=GRIDS, ids=lambda p: "x".join(map(str, p[:3])))
def pair(request, built):
    mx, my, n, Lx, Ly = request.param
    og = SMPMGrid(mx, my, n, Lx, Ly)
    return og, SchurSystem(og), og.assemble_L(), Grid(mx, my, n, Lx, Ly)


def columns(og, R, seed):
    F = np.stack([inputs.white_noise(og.r, seed + k) for k in range(R)])
    Gs = np.random.default_rng(seed).standard_normal((R, og.kp))
    return F, Gs


@pytest.mark.parametrize("flags", [0, B.FLAG_NO_SMEM_RESIDENCY], ids=["resident", "global"])
@pytest.mark.parametrize("precond", [1, 2])
@pytest.mark.parametrize("R", [2, 3, 8, 16])
def test_lockstep_columns_match_oracle(pair, R, precond, flags):
    og, osys, Lm, lg = pair
    lg.factor(tol=1e-12, precond=precond, flags=flags)
    F, Gs = columns(og, R, 100 * R + precond)
    U = torch.zeros((R, og.r), dtype=torch.float64, device="cuda")
    reps = lg.solve(dev(F), U, g=dev(Gs), nrhs=R)
    Uh = host(U)
    alg = methods.algorithm2 if precond == 1 else methods.algorithm3
    for k in range(0, R, max(1, R // 4)):            # a sample of the columns against the oracle
        b = og.rhs(F[k], Gs[k])
        ud = methods.direct_solve(og, Lm, osys.u_L, b)
        uo, info = alg(osys, b, tol=1e-12, restart=50)
        assert reps[k]["converged"] == 1, (k, reps[k])
        assert rel(Uh[k], ud) < 1e-10, (k, rel(Uh[k], ud))
        assert rel(Uh[k], uo) < 1e-10, (k, rel(Uh[k], uo))
        assert abs(reps[k]["iterations"] - info["iterations"]) <= 1, (k, reps[k], info["iterations"])
        assert reps[k]["schur_relres"] < 1e-10
    # every column against the library's one-at-a-time solve
    lg.factor(tol=1e-12, precond=precond, flags=flags | B.FLAG_NO_LOCKSTEP)
    U1 = torch.zeros_like(U)
    reps1 = lg.solve(dev(F), U1, g=dev(Gs), nrhs=R)
    U1h = host(U1)
    for k in range(R):
        assert rel(Uh[k], U1h[k]) < 1e-10, k
        assert abs(reps[k]["iterations"] - reps1[k]["iterations"]) <= 1, (k, reps[k], reps1[k])


def test_zero_column_and_mixed_counts(pair):
    """A zero right-hand side between two others: it stops at once (no
    iterations, u = 0) while the others run to tol."""
    og, osys, Lm, lg = pair
    lg.factor(tol=1e-12)
    F, _ = columns(og, 3, 7)
    F[1] = 0.0
    U = torch.full((3, og.r), 5.0, dtype=torch.float64, device="cuda")
    reps = lg.solve(dev(F), U, nrhs=3)
    Uh = host(U)
    assert reps[1]["iterations"] == 0 and reps[1]["converged"] == 1 and np.abs(Uh[1]).max() == 0.0
    for k in (0, 2):
        ud = methods.direct_solve(og, Lm, osys.u_L, F[k])
        assert reps[k]["converged"] == 1 and rel(Uh[k], ud) < 1e-10


def test_columns_stopped_at_maxit(built):
    """maxit reached in every column (across a restart): each column holds
    the solution assembled from its last iterate, the oracle's Algorithm 3
    stopped at the same step."""
    og = SMPMGrid(4, 3, 6)
    osys = SchurSystem(og)
    lg = Grid(4, 3, 6)
    lg.factor(tol=1e-12, maxit=7, restart=4)
    F, _ = columns(og, 4, 61)
    U = torch.zeros((4, og.r), dtype=torch.float64, device="cuda")
    reps = lg.solve(dev(F), U, nrhs=4, allow_notconv=True)
    Uh = host(U)
    for k in range(4):
        uo, info = methods.algorithm3(osys, F[k], tol=1e-12, restart=4, maxit=7)
        assert reps[k]["status"] == B.SMPM_ENOTCONV and reps[k]["converged"] == 0 and reps[k]["iterations"] == 7
        assert rel(Uh[k], uo) < 1e-10, k


@pytest.mark.parametrize("R", [2, 5, 8])
def test_lockstep_mixed_precision_columns(pair, R):
    """FP32 inner lockstep GMRES inside per-column FP64 iterative refinement:
    every column within 1e-9 of the exact discrete solution (the oracle's
    direct solve), as the one-at-a-time mixed solve."""
    og, osys, Lm, lg = pair
    lg.factor(tol=1e-11, precision=1)
    F, Gs = columns(og, R, 300 + R)
    U = torch.zeros((R, og.r), dtype=torch.float64, device="cuda")
    reps = lg.solve(dev(F), U, g=dev(Gs), nrhs=R)
    Uh = host(U)
    for k in range(R):
        b = og.rhs(F[k], Gs[k])
        ud = methods.direct_solve(og, Lm, osys.u_L, b)
        assert reps[k]["converged"] == 1 and reps[k]["refinements"] >= 1, (k, reps[k])
        assert rel(Uh[k], ud) < 1e-9, (k, rel(Uh[k], ud))
    lg.factor(tol=1e-11, precision=1, flags=B.FLAG_NO_LOCKSTEP)
    U1 = torch.zeros_like(U)
    lg.solve(dev(F), U1, g=dev(Gs), nrhs=R)
    U1h = host(U1)
    for k in range(R):
        assert rel(Uh[k], U1h[k]) < 1e-9, k
