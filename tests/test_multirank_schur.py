"""The element-tile partition (smpm_partition_tile / smpm_partition_halo)
driving Algorithm 3 over gloo ranks on the CPU: every operator of the
sharded solve (S, M^-1, P, Q, all-reduced dots) and the whole deflated GMRES
against the oracle's global ones, on 2, 3 and 4 ranks, a uniform and a graded
grid.  The tiles and halo lists are also checked on their own: they cover
every element once, each cut has matching lists on its two sides, and the
halo is n slots per cut interface."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from paper_1601_03432_gb300 import _binding as B, inputs  # noqa: E402
from oracle.smpm import SMPMGrid  # noqa: E402
from oracle.schur import SchurSystem  # noqa: E402
from oracle import methods  # noqa: E402
from oracle.gmres import gmres  # noqa: E402

UNIFORM = dict(mx=6, my=5, n=5, Lx=1.2, Ly=1.0)
GRADED = dict(mx=4, my=3, n=6, xs=[0.0, 0.2, 0.5, 1.0, 1.3], ys=[0.0, 0.35, 0.5, 1.1])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _grids(spec):
    kw = {k: spec[k] for k in ("Lx", "Ly", "xs", "ys") if k in spec}
    return (SMPMGrid(spec["mx"], spec["my"], spec["n"], **kw),
            B.Grid(spec["mx"], spec["my"], spec["n"], **kw))


@pytest.mark.parametrize("px,py", [(1, 1), (2, 1), (3, 2), (2, 3), (6, 5)])
def test_tiles_and_halos_partition_the_grid(px, py):
    og, lg = _grids(UNIFORM)
    n, M = og.n, 4 * og.n
    owner = -np.ones(og.nel, dtype=int)
    for rank in range(px * py):
        t = lg.partition_tile(px, py, rank)
        for iy in range(t["iy0"], t["iy1"]):
            for ix in range(t["ix0"], t["ix1"]):
                assert owner[iy * og.mx + ix] < 0
                owner[iy * og.mx + ix] = rank
        assert t["nel_owned"] == (t["ix1"] - t["ix0"]) * (t["iy1"] - t["iy0"])
        for side in range(4):
            peer = t["peers"][side]
            if peer < 0:
                assert t["halo"][side] == 0
                with pytest.raises(B.SmpmError):
                    lg.partition_halo(px, py, rank, side)
                continue
            own, facing = lg.partition_halo(px, py, rank, side)
            assert len(own) == t["halo"][side] and len(own) % n == 0
            p_own, p_facing = lg.partition_halo(px, py, peer, side ^ 1)
            assert np.array_equal(own, p_facing) and np.array_equal(facing, p_own)
            for s_own, s_fac in zip(own, facing):       # slot pairs facing each other across the cut
                e, F, t_ = s_own // M, (s_own % M) // n, s_own % n
                assert og.neighbour(e, F) == s_fac // M and (s_fac % M) // n == (F ^ 1) and s_fac % n == t_
                assert owner[e] == rank
    assert np.all(owner >= 0)
    # balanced tiles: sizes differ by at most one element row or column
    widths = {lg.partition_tile(px, py, r)["ix1"] - lg.partition_tile(px, py, r)["ix0"] for r in range(px)}
    assert max(widths) - min(widths) <= 1
    with pytest.raises(B.SmpmError):
        lg.partition_tile(og.mx + 1, 1, 0)


def _worker(rank, world, port, spec, px, py, inputs_, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from dist_schur import ShardedSchur
    _, lg = _grids(spec)
    lg.factor_host_only(tol=1e-11)
    sh = ShardedSchur(lg, px, py, rank)
    v, bS = inputs_["v"], inputs_["bS"]
    res = {"S": sh.gather(sh.apply_S(v)), "Minv": sh.gather(sh.apply_Minv(v)),
           "P": sh.gather(sh.apply_P(v)), "Q": sh.gather(sh.apply_Q(v)), "dot": sh.dot(v, bS)}
    x, its = sh.algorithm3(bS, tol=1e-11)
    res["x"], res["its"], res["sent"] = sh.gather(x), its, sh.exchanged
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("spec,px,py", [(UNIFORM, 2, 1), (UNIFORM, 3, 1), (UNIFORM, 2, 2), (GRADED, 2, 2)],
                         ids=["uniform-2x1", "uniform-3x1", "uniform-2x2", "graded-2x2"])
def test_sharded_algorithm3_matches_oracle(spec, px, py):
    og, lg = _grids(spec)
    lg.factor_host_only(tol=1e-11)   # builds the library before the ranks start
    osys = SchurSystem(og)
    rng = np.random.default_rng(61)
    v = og.to_padded(rng.standard_normal(og.k))
    b = methods.project_rhs(osys, og.rhs(inputs.white_noise(og.r, 62)))
    bSc = methods.schur_rhs_projected(osys, b)
    op = lambda q: osys.apply_P(osys.apply_S(osys.apply_Minv(q)))
    y, info = gmres(op, osys.apply_P(bSc), 1e-11, 50, 1000)
    x_ref = osys.apply_Q(osys.apply_Minv(y)) + osys.Z @ osys.coarse_solve(osys.Z.T @ bSc)
    world = px * py
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), spec, px, py, {"v": v, "bS": og.to_padded(bSc)}, out),
             nprocs=world, join=True)
    vc = og.from_padded(v)
    refs = {"S": osys.apply_S(vc), "Minv": osys.apply_Minv(vc), "P": osys.apply_P(vc), "Q": osys.apply_Q(vc)}
    for rank in range(world):
        r = out[rank]
        for name, ref in refs.items():
            got = og.from_padded(r[name])
            assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref), (rank, name)
        assert r["dot"] == pytest.approx(vc @ bSc, rel=1e-12)
        x = og.from_padded(r["x"])
        assert np.linalg.norm(osys.apply_S(x) - bSc) <= 1e-9 * np.linalg.norm(bSc)
        assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
        assert abs(r["its"] - info["iterations"]) <= 1, (r["its"], info["iterations"])
        assert r["sent"] > 0
