"""Failure paths of the solve, in forms that fault and hang nothing:

* ENOTCONV: maxit reached; u holds the solution assembled from the last
  iterate, which must equal the oracle's Algorithm 3 stopped at the same step
  count (also across a restart).
* EBREAKDOWN: a tolerance below round-off on a small grid; the Krylov space
  becomes invariant before the estimate reaches tol.  The oracle's GMRES
  reports the same breakdown, and u is then the exact discrete solution.
* ETIMEOUT: the device-side barrier waits are given a poll limit so small
  that real waits run out; every CTA unwinds, the call returns ETIMEOUT, and
  the same handle solves correctly once the default limit is back.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1601_03432_gb300 import Grid, Batch, inputs, factor_many
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


@pytest.mark.parametrize("maxit,restart", [(1, 50), (3, 2), (7, 4)])
def test_notconv_returns_the_last_iterate(built, maxit, restart):
    og = SMPMGrid(4, 3, 6)
    osys = SchurSystem(og)
    lg = Grid(4, 3, 6)
    lg.factor(tol=1e-12, maxit=maxit, restart=restart)
    f = inputs.white_noise(og.r, 51)
    u = torch.zeros(og.r, dtype=torch.float64, device="cuda")
    rep = lg.solve(dev(f), u, allow_notconv=True)[0]
    assert rep["status"] == B.SMPM_ENOTCONV and rep["converged"] == 0 and rep["iterations"] == maxit, rep
    uo, info = methods.algorithm3(osys, f, tol=1e-12, restart=restart, maxit=maxit)
    assert not info["converged"] and info["iterations"] == maxit
    assert rel(host(u), uo) < 1e-10


def test_breakdown_below_roundoff(built):
    og = SMPMGrid(2, 2, 3, 1.5, 1.0)
    osys = SchurSystem(og)
    lg = Grid(2, 2, 3, 1.5, 1.0)
    lg.factor(tol=1e-30)
    f = inputs.white_noise(og.r, 52)
    u = torch.zeros(og.r, dtype=torch.float64, device="cuda")
    rep = lg.solve(dev(f), u, allow=(B.SMPM_EBREAKDOWN,))[0]
    assert rep["status"] == B.SMPM_EBREAKDOWN and rep["converged"] == 0, rep
    uo, info = methods.algorithm3(osys, f, tol=1e-30)
    assert info["breakdown"] and not info["converged"]
    # where round-off ends the Krylov process differs between CGS2 and MGS:
    # the CUDA path (CGS2) stays within the dimension of the space; the
    # oracle's MGS may run a few steps past it on round-off
    assert rep["iterations"] <= og.k and info["iterations"] <= og.k + 8
    ud = methods.direct_solve(og, og.assemble_L(), osys.u_L, f)
    assert rel(host(u), ud) < 1e-10


def test_barrier_timeout_unwinds_and_context_survives(built):
    og = SMPMGrid(16, 16, 8)
    osys = SchurSystem(og)
    lg = Grid(16, 16, 8)
    lg.factor(tol=1e-12)
    f = inputs.white_noise(og.r, 53)
    ud = methods.direct_solve(og, og.assemble_L(), osys.u_L, f)
    u = torch.zeros(og.r, dtype=torch.float64, device="cuda")
    try:
        B.set_barrier_spin_limit(1)
        with pytest.raises(B.SmpmError) as ei:
            lg.solve(dev(f), u)
        assert ei.value.status == B.SMPM_ETIMEOUT
    finally:
        B.set_barrier_spin_limit(0)
    rep = lg.solve(dev(f), u)[0]
    assert rep["converged"] == 1 and rel(host(u), ud) < 1e-10


def test_batch_barrier_timeout_unwinds(built):
    probs = [(4, 3, 6), (5, 4, 7), (3, 3, 8)]
    grids = [Grid(*p) for p in probs]
    factor_many(grids, tol=1e-12)
    refs, fs = [], []
    for gr, p in zip(grids, probs):
        og = SMPMGrid(*p)
        f = inputs.white_noise(og.r, 54)
        fs.append(f)
        refs.append(methods.direct_solve(og, og.assemble_L(), SchurSystem(og).u_L, f))
    b = Batch(grids, [1] * len(grids), team_size=8)
    fd = dev(np.concatenate(fs))
    u = torch.zeros_like(fd)
    try:
        B.set_barrier_spin_limit(1)
        with pytest.raises(B.SmpmError) as ei:
            b.solve(fd, u)
        assert ei.value.status == B.SMPM_ETIMEOUT
    finally:
        B.set_barrier_spin_limit(0)
    u.zero_()
    b.solve(fd, u)
    uh, o = host(u), 0
    for ref in refs:
        assert rel(uh[o:o + ref.size], ref) < 1e-10
        o += ref.size
    b.close()
