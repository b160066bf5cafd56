"""GPU parity of batched solves (smpm_batch_*): many right-hand sides of
uneven grids in one persistent launch, against the oracle's direct solve and
against the single-grid solves of the same handles.

Tolerances as for single solves: relative L2 error 1e-10 (FP64) and 1e-9
(mixed precision) against the exact discrete solution; iteration counts
within one of the single solves (team sizes change the order of the FP64
atomic sums, nothing else)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1601_03432_gb300 import Batch, Grid, factor_many, inputs
from paper_1601_03432_gb300 import _binding as B
from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import methods

PROBLEMS = [(3, 2, 5, 2), (4, 4, 6, 1), (2, 3, 8, 3), (5, 4, 7, 2), (6, 3, 4, 1)]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def built():
    from paper_1601_03432_gb300.build import build
    build()
    assert torch.cuda.is_available()


def make_inputs(problems, seed, with_g=True):
    rng = np.random.default_rng(seed)
    fs, gs, refs = [], [], []
    for (mx, my, n, k) in problems:
        og = SMPMGrid(mx, my, n)
        osys = SchurSystem(og)
        Lm = og.assemble_L()
        for _ in range(k):
            f = rng.standard_normal(og.r)
            g = rng.standard_normal(og.kp) if with_g else np.zeros(og.kp)
            fs.append(f)
            gs.append(g)
            refs.append(methods.direct_solve(og, Lm, osys.u_L, og.rhs(f, g)))
    return fs, gs, refs


def packed(arrs):
    return torch.as_tensor(np.concatenate(arrs), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("team", [1, 2, 4, 19, 152])
@pytest.mark.parametrize("graph", [True, False], ids=["graph", "nograph"])
def test_batch_matches_direct_solve(built, precision, team, graph):
    grids = [Grid(mx, my, n) for (mx, my, n, _) in PROBLEMS]
    for g in grids:
        g.factor(tol=1e-12 if precision == 0 else 1e-11, precision=precision)
    fs, gs, refs = make_inputs(PROBLEMS, 5)
    b = Batch(grids, [k for *_, k in PROBLEMS], team_size=team, use_graph=graph)
    assert b.info()["team_size"] == team
    f, g = packed(fs), packed(gs)
    u = torch.zeros_like(f)
    for rep_round in range(2):  # the second call replays the graph
        u.zero_()
        reps = b.solve(f, u, g=g)
        uh = u.cpu().numpy()
        o = 0
        for i, ref in enumerate(refs):
            got = uh[o:o + ref.size]
            o += ref.size
            assert reps[i]["converged"] == 1
            assert rel(got, ref) < (1e-10 if precision == 0 else 1e-9), (i, reps[i], rel(got, ref))
    # same iteration counts as the single-grid solves (within one)
    i = 0
    for gr, (_, _, _, k) in zip(grids, PROBLEMS):
        for _ in range(k):
            fi = torch.as_tensor(fs[i], dtype=torch.float64, device="cuda")
            gi = torch.as_tensor(gs[i], dtype=torch.float64, device="cuda")
            ui = torch.zeros_like(fi)
            r1 = gr.solve(fi, ui, g=gi)[0]
            assert abs(r1["iterations"] - reps[i]["iterations"]) <= 1, (i, r1, reps[i])
            i += 1
    b.close()


def test_batch_without_g_and_autotune(built):
    probs = [(4, 5, 6, 2), (3, 3, 9, 1), (7, 2, 5, 3)]
    grids = [Grid(mx, my, n) for (mx, my, n, _) in probs]
    for gr in grids:
        gr.factor(tol=1e-11, precision=1)
    fs, _, refs = make_inputs(probs, 8, with_g=False)
    b = Batch(grids, [k for *_, k in probs])
    f = packed(fs)
    u = torch.zeros_like(f)
    chosen, ms = b.autotune(f, u, candidates=(2, 8, 38))
    assert chosen in (2, 8, 38) and ms[chosen] > 0
    u.zero_()
    b.solve(f, u)
    uh = u.cpu().numpy()
    o = 0
    for ref in refs:
        assert rel(uh[o:o + ref.size], ref) < 1e-9
        o += ref.size


def test_batch_precision_override(built):
    """Handles factored for mixed precision, solved as a batch in FP64 and in
    mixed precision (the factors hold both)."""
    probs = [(4, 3, 6, 2), (3, 5, 8, 1)]
    grids = [Grid(mx, my, n) for (mx, my, n, _) in probs]
    factor_many(grids, tol=1e-12, precision=1)
    fs, gs, refs = make_inputs(probs, 12)
    f, g = packed(fs), packed(gs)
    for prec, bound in ((0, 1e-10), (1, 1e-9)):
        b = Batch(grids, [k for *_, k in probs], precision=prec)
        u = torch.zeros_like(f)
        reps = b.solve(f, u, g=g)
        assert all(r["refinements"] == 0 for r in reps) == (prec == 0)
        uh = u.cpu().numpy()
        o = 0
        for ref in refs:
            assert rel(uh[o:o + ref.size], ref) < bound
            o += ref.size
        b.close()


def test_batch_config4_sample(built):
    """The first 12 problems of the seeded uneven config-4 batch (mixed
    precision, 1e-10): the right-hand sides of the four smallest problems
    (up to three each) against the oracle's direct bordered solve (1e-9, the
    bound after refinement), and every right-hand side against the
    single-grid solve of the same handle."""
    probs = inputs.uneven_batch(512, seed=7)[:12]
    grids = [Grid(mx, my, n) for (mx, my, n, k) in probs]
    factor_many(grids, tol=1e-10, precision=1)
    fs = []
    for gr, (mx, my, n, k) in zip(grids, probs):
        x, y = gr.node_coords()
        for j in range(k):
            fs.append(inputs.fourier_rhs(x, y, seed=1000 + j)[0])
    b = Batch(grids, [p[3] for p in probs])
    f = packed(fs)
    u = torch.zeros_like(f)
    reps = b.solve(f, u)
    assert all(r["converged"] == 1 for r in reps)
    uh = u.cpu().numpy()
    small = sorted(range(len(probs)), key=lambda q: probs[q][0] * probs[q][1] * probs[q][2] ** 2)[:4]
    o, i = 0, 0
    for q, (gr, p) in enumerate(zip(grids, probs)):
        og = SMPMGrid(p[0], p[1], p[2]) if q in small else None
        Lm = og.assemble_L() if og is not None else None
        uL = SchurSystem(og).u_L if og is not None else None
        for j in range(p[3]):
            fi = torch.as_tensor(fs[i], dtype=torch.float64, device="cuda")
            ui = torch.zeros_like(fi)
            gr.solve(fi, ui)
            assert rel(uh[o:o + gr.r], ui.cpu().numpy()) < 1e-8
            if og is not None and j < 3:
                ud = methods.direct_solve(og, Lm, uL, fs[i])
                assert rel(uh[o:o + gr.r], ud) < 1e-9, (q, j, rel(uh[o:o + gr.r], ud))
            o += gr.r
            i += 1


@pytest.mark.parametrize("kind", [0, 1], ids=["ring", "warp"])
def test_batched_apply_matches_single_grid_apply(built, kind):
    """y_p = S_p v_p for all problems in one launch, FP64 against the oracle's
    S and FP32 against it to FP32 round-off; uneven n (different element
    matrix sizes in one launch)."""
    probs = [(3, 2, 5, 1), (4, 4, 9, 1), (2, 5, 12, 1), (6, 3, 7, 1)]
    grids = [Grid(mx, my, n) for (mx, my, n, _) in probs]
    factor_many(grids, precision=1)
    b = Batch(grids, [1] * len(grids))
    b.set_apply_kernel(kind)
    rng = np.random.default_rng(17)
    ogs = [SMPMGrid(mx, my, n) for (mx, my, n, _) in probs]
    vs = [rng.standard_normal(og.k) for og in ogs]
    vp = np.concatenate([og.to_padded(v) for og, v in zip(ogs, vs)])
    assert vp.size == b.v_len()
    v64 = torch.as_tensor(vp, dtype=torch.float64, device="cuda")
    y64 = torch.full_like(v64, 3.0)
    b.apply_schur(v64, y64)
    v32 = v64.float()
    y32 = torch.full_like(v32, 3.0)
    b.apply_schur32(v32, y32)
    h64, h32 = y64.cpu().numpy(), y32.double().cpu().numpy()
    o = 0
    for og, v in zip(ogs, vs):
        ref = SchurSystem(og).apply_S(v)
        assert rel(og.from_padded(h64[o:o + og.kp]), ref) < 1e-12
        assert rel(og.from_padded(h32[o:o + og.kp]), ref) < 1e-5
        pad = np.setdiff1d(np.arange(og.kp), og.padded_index)
        assert np.all(h64[o + pad] == 0) and np.all(h32[o + pad] == 0)
        o += og.kp


@pytest.mark.parametrize("precision,bound", [(0, 1e-10), (1, 1e-9)], ids=["fp64", "mixed"])
def test_batch_lockstep_groups_match_one_at_a_time(built, precision, bound):
    """Problems with several right-hand sides run as lockstep groups inside
    the batched launch (up to 16 columns per group; 19 right-hand sides make
    a group of 16 and a group of 3; 1 stays a single task).  Every column
    matches the oracle's direct solve and the batch whose handles ask for one
    right-hand side at a time (SMPM_FLAG_NO_LOCKSTEP)."""
    probs = [(4, 3, 6, 5), (5, 4, 7, 19), (3, 3, 8, 1), (6, 5, 5, 2)]
    fs, gs, refs = make_inputs(probs, 31)
    f, g = packed(fs), packed(gs)
    sols = []
    for flags in (0, B.FLAG_NO_LOCKSTEP):
        grids = [Grid(mx, my, n) for (mx, my, n, _) in probs]
        factor_many(grids, tol=1e-12 if precision == 0 else 1e-11, precision=precision, flags=flags)
        b = Batch(grids, [k for *_, k in probs], team_size=8)
        u = torch.zeros_like(f)
        reps = b.solve(f, u, g=g)
        assert all(r["converged"] == 1 for r in reps), reps
        uh = u.cpu().numpy()
        o = 0
        for ref in refs:
            assert rel(uh[o:o + ref.size], ref) < bound
            o += ref.size
        sols.append(uh)
        b.close()
    assert rel(sols[0], sols[1]) < bound
