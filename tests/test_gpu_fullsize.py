"""Parity at full size against stored oracle references.

The oracle's Algorithm 3 takes minutes of setup at these sizes (sparse LU of
the bordered S^T for u_S), so its solutions were computed once by
tests/golden/make_fullsize_refs.py (which calls only the oracle and the seeded
input generators) and stored as every 997th entry plus the L2 norm of the
whole zero-mean solution.  The GPU solution is compared on those entries
(relative L2 over the sample) and in norm:

* 32 x 32 elements, n = 24, Fourier right-hand sides of seeds 1000 (oracle
  to 1e-12) and 1001 (oracle to 1e-11), solved together (lockstep) to 1e-11:
  FP64 within 1e-10 of the oracle, mixed precision (FP32 inner GMRES, FP64
  refinement) within 1e-9; FP64 iteration counts within one of the oracle's
  at the same tolerance.
* 48 x 48 elements, n = 16, Fourier right-hand side of seed 6 to 1e-11:
  FP64 within 1e-10.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1601_03432_gb300 import Grid, inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_ref(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        lines = [ln for ln in fh if not ln.startswith("#")]
    head = lines[0].split()
    meta = {head[i]: float(head[i + 1]) for i in range(0, len(head), 2)}
    norm = float(lines[1].split()[1])
    idx, val = [], []
    for ln in lines[2:]:
        i, v = ln.split()
        idx.append(int(i))
        val.append(float(v))
    return meta, norm, np.array(idx), np.array(val)


def check(u, ref, bound):
    meta, norm, idx, val = ref
    assert u.size == int(meta["r"])
    err = np.linalg.norm(u[idx] - val) / np.linalg.norm(val)
    assert err < bound, err
    assert abs(np.linalg.norm(u) - norm) <= bound * norm


@pytest.fixture(scope="module")
def built():
    from paper_1601_03432_gb300.build import build
    build()
    assert torch.cuda.is_available()


@pytest.mark.slow
@pytest.mark.parametrize("prec,bound", [(0, 1e-10), (1, 1e-9)], ids=["fp64", "mixed"])
def test_config3_against_oracle(built, prec, bound):
    seeds = (1000, 1001)
    refs = [read_ref("config3_32x32_n24_fourier%d.txt" % s) for s in seeds]
    lg = Grid(32, 32, 24)
    lg.factor(tol=1e-11, precision=prec)
    x, y = lg.node_coords()
    F = np.stack([inputs.fourier_rhs(x, y, seed=s)[0] for s in seeds])
    U = torch.zeros((2, lg.r), dtype=torch.float64, device="cuda")
    reps = lg.solve(torch.as_tensor(F, device="cuda"), U, nrhs=2)
    torch.cuda.synchronize()
    Uh = U.cpu().numpy()
    for k, ref in enumerate(refs):
        assert reps[k]["converged"] == 1, reps[k]
        check(Uh[k], ref, bound)
        if prec == 0 and ref[0]["tol"] == 1e-11:
            assert abs(reps[k]["iterations"] - int(ref[0]["iterations"])) <= 1, (reps[k], ref[0])
    if prec == 0:   # seed 1000 alone at the oracle's 1e-12
        u = torch.zeros(lg.r, dtype=torch.float64, device="cuda")
        rep = lg.solve(torch.as_tensor(F[0], device="cuda"), u, tol=1e-12)[0]
        torch.cuda.synchronize()
        assert rep["converged"] == 1
        check(u.cpu().numpy(), refs[0], bound)
        # at 1e-12 both solvers are close to what FP64 attains on this grid, and
        # where each crosses the line differs by up to two steps
        assert abs(rep["iterations"] - int(refs[0][0]["iterations"])) <= 2, (rep, refs[0][0])


@pytest.mark.slow
def test_config5_forward_against_oracle(built):
    ref = read_ref("config5_48x48_n16_fourier6.txt")
    lg = Grid(48, 48, 16)
    lg.factor(tol=1e-11)
    x, y = lg.node_coords()
    f, _ = inputs.fourier_rhs(x, y, seed=6)
    u = torch.zeros(lg.r, dtype=torch.float64, device="cuda")
    rep = lg.solve(torch.as_tensor(f, device="cuda"), u)[0]
    torch.cuda.synchronize()
    assert rep["converged"] == 1
    check(u.cpu().numpy(), ref, 1e-10)
    assert abs(rep["iterations"] - int(ref[0]["iterations"])) <= 1, (rep, ref[0])
