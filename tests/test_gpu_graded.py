"""Graded grids on the GPU path (Sec. 1.2: elements of their own sizes; the
column widths and row heights differ), through the C ABI, against the oracle
on the same seeded inputs.

Every element then carries distinct factors, tau_F and p_F differ across an
interface, and the deflation vectors z_j are B 1 restricted to each interface
(divided by the mean of its two sides), the indicators of Sec. 2 on a uniform
grid.  Covered: the single operators, the solve for Algorithms 1-3 in every
GMRES layout, mixed precision, the adjoint, lockstep columns, the class-shared
apply, a batch mixing graded and uniform grids, and a wall-clustered grid of
24 x 24 elements.  Bounds as for uniform grids: operators 1e-12 relative,
FP64 solutions 1e-10 against the direct solve and the oracle's algorithm,
iteration counts within one, mixed precision 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1601_03432_gb300 import Grid, Batch, inputs
from paper_1601_03432_gb300 import _binding as B
from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import methods, adjoint

GRADED = {
    "jagged4x3": ([0.0, 0.2, 0.5, 1.0, 1.3], [0.0, 0.35, 0.5, 1.1], 6),
    "cols3x3": ([0.0, 0.3, 0.45, 1.0], [0.0, 0.5, 1.0, 1.5], 5),
    "wall8x6": (list(inputs.clustered_edges(8, 1.0, 2.0)), list(inputs.clustered_edges(6, 0.5, 1.5)), 7),
    "jitter7x5": (list(inputs.jittered_edges(7, 1.4, 3)), list(inputs.jittered_edges(5, 1.0, 4)), 5),
}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def zeros(n):
    return torch.zeros(n, dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def built():
    from paper_1601_03432_gb300.build import build
    build()
    assert torch.cuda.is_available()


def make(xs, ys, n):
    og = SMPMGrid(len(xs) - 1, len(ys) - 1, n, xs=xs, ys=ys)
    lg = Grid(og.mx, og.my, n, xs=xs, ys=ys)
    return og, lg


@pytest.fixture(scope="module", params=list(GRADED), ids=list(GRADED))
def gpair(request, built):
    og, lg = make(*GRADED[request.param])
    osys = SchurSystem(og)
    assert osys.coarse_singular and np.abs(osys.zweights - 1).max() > 1e-3
    lg.factor(tol=1e-12)
    return og, osys, lg


def test_graded_geometry_matches_oracle(gpair):
    og, osys, lg = gpair
    x, y = lg.node_coords()
    ox, oy = og.coords()
    np.testing.assert_allclose(x, ox, atol=1e-14)
    np.testing.assert_allclose(y, oy, atol=1e-14)
    np.testing.assert_allclose(lg.node_mass(), og.mass(), rtol=1e-13)


def test_graded_operators(gpair):
    og, osys, lg = gpair
    rng = np.random.default_rng(31)
    v = rng.standard_normal(og.k)
    vp = dev(og.to_padded(v))
    out = zeros(og.kp)
    lg.apply_schur(vp, out)
    assert rel(og.from_padded(host(out)), osys.apply_S(v)) < 1e-12
    lg.apply_precond(vp, out)
    assert rel(og.from_padded(host(out)), osys.apply_Minv(v)) < 1e-12
    lg.apply_deflation(vp, out)
    assert rel(og.from_padded(host(out)), osys.apply_P(v)) < 1e-11
    lg.apply_deflation_q(vp, out)
    assert rel(og.from_padded(host(out)), osys.apply_Q(v)) < 1e-11
    b = rng.standard_normal(og.r)
    lg.schur_rhs(dev(b), out)
    assert rel(og.from_padded(host(out)), osys.schur_rhs(b)) < 1e-12
    u = zeros(og.r)
    lg.recover(dev(b), vp, u)
    assert rel(host(u), osys.recover(b, v)) < 1e-12
    uL, uS, uC = zeros(og.r), zeros(og.kp), zeros(og.d)
    lg.null_vectors(uL, uS, uC)
    for got, ref in ((host(uL), osys.u_L), (og.from_padded(host(uS)), osys.u_S), (host(uC), osys.u_C)):
        assert np.linalg.norm(got * np.sign(got @ ref) - ref) < 1e-12


def test_graded_class_shared_apply(gpair):
    og, osys, lg = gpair
    v = np.random.default_rng(32).standard_normal(og.k)
    out = zeros(og.kp)
    lg.apply_schur_class(dev(og.to_padded(v)), out)
    assert rel(og.from_padded(host(out)), osys.apply_S(v)) < 1e-12


@pytest.mark.parametrize("flags", [0, 2, 8], ids=["smem", "stream", "warps"])
@pytest.mark.parametrize("precond", [0, 1, 2])
def test_graded_solve_matches_oracle(gpair, precond, flags):
    og, osys, lg = gpair
    f = inputs.white_noise(og.r, 33)
    gslots = np.random.default_rng(34).standard_normal(og.kp)
    b = og.rhs(f, gslots)
    ud = methods.direct_solve(og, og.assemble_L(), osys.u_L, b)
    alg = [methods.algorithm1, methods.algorithm2, methods.algorithm3][precond]
    uo, info = alg(osys, b, tol=1e-12, restart=50)
    lg.factor(precond=precond, tol=1e-12, flags=flags)
    u = zeros(og.r)
    rep = lg.solve(dev(f), u, g=dev(gslots), tol=1e-12)[0]
    uh = host(u)
    assert rep["converged"] == 1
    assert rel(uh, ud) < 1e-10
    assert rel(uh, uo) < 1e-10
    assert abs(rep["iterations"] - info["iterations"]) <= 1, (rep, info["iterations"])
    lg.factor(tol=1e-12)


def test_graded_mixed_precision(gpair):
    og, osys, lg = gpair
    f = inputs.white_noise(og.r, 35)
    ud = methods.direct_solve(og, og.assemble_L(), osys.u_L, og.rhs(f))
    lg.factor(precision=1, tol=1e-11)
    u = zeros(og.r)
    rep = lg.solve(dev(f), u)[0]
    assert rep["converged"] == 1 and rel(host(u), ud) < 1e-9
    lg.factor(tol=1e-12)


def test_graded_adjoint(gpair):
    og, osys, lg = gpair
    lg.factor(tol=1e-12, flags=B.FLAG_ADJOINT)
    gbar = inputs.white_noise(og.r, 36)
    ref = adjoint.adjoint_direct(og, og.assemble_L(), osys.u_L, gbar)
    _, refg = adjoint.grad_f_g(og, ref)
    gf, gg = zeros(og.r), zeros(og.kp)
    rep = lg.solve_adjoint(dev(gbar), gf, gg)[0]
    assert rep["converged"] == 1
    assert rel(host(gf), ref) < 1e-9
    assert rel(host(gg), refg) < 1e-9
    lg.factor(tol=1e-12)


@pytest.mark.parametrize("R", [3, 8])
def test_graded_lockstep_columns(gpair, R):
    og, osys, lg = gpair
    Lm = og.assemble_L()
    F = np.stack([inputs.white_noise(og.r, 40 + k) for k in range(R)])
    Gs = np.random.default_rng(41).standard_normal((R, og.kp))
    u = zeros(R * og.r)
    reps = lg.solve(dev(F.ravel()), u, g=dev(Gs.ravel()), nrhs=R, tol=1e-12)
    uh = host(u).reshape(R, og.r)
    for k in range(R):
        ud = methods.direct_solve(og, Lm, osys.u_L, og.rhs(F[k], Gs[k]))
        assert reps[k]["converged"] == 1 and rel(uh[k], ud) < 1e-10, (k, reps[k])


def test_graded_and_uniform_in_one_batch(built):
    problems = [("jagged4x3", 2), (None, 1), ("wall8x6", 3), ("jitter7x5", 1)]
    grids, ogs, ks = [], [], []
    for name, k in problems:
        if name is None:
            og, lg = SMPMGrid(3, 2, 5, 1.5, 0.75), Grid(3, 2, 5, 1.5, 0.75)
        else:
            og, lg = make(*GRADED[name])
        lg.factor(tol=1e-12)
        grids.append(lg)
        ogs.append(og)
        ks.append(k)
    rng = np.random.default_rng(42)
    fs, gs, refs = [], [], []
    for og, k in zip(ogs, ks):
        osys = SchurSystem(og)
        Lm = og.assemble_L()
        for _ in range(k):
            f, g = rng.standard_normal(og.r), rng.standard_normal(og.kp)
            fs.append(f)
            gs.append(g)
            refs.append(methods.direct_solve(og, Lm, osys.u_L, og.rhs(f, g)))
    b = Batch(grids, ks, team_size=4)
    f, g = dev(np.concatenate(fs)), dev(np.concatenate(gs))
    u = torch.zeros_like(f)
    reps = b.solve(f, u, g=g)
    uh, o = host(u), 0
    for i, ref in enumerate(refs):
        assert reps[i]["converged"] == 1 and rel(uh[o:o + ref.size], ref) < 1e-10, (i, reps[i])
        o += ref.size
    b.close()


def test_wall_clustered_grid_24x24(built):
    """24 x 24 elements, n = 10, tanh-clustered toward all four walls (element
    sizes spanning a factor of about 12), Fourier f and Neumann data g."""
    xs = inputs.clustered_edges(24, 1.0, 2.0)
    og, lg = make(list(xs), list(xs), 10)
    osys = SchurSystem(og)
    x, y = og.coords()
    f, _ = inputs.fourier_rhs(x, y, seed=1002)
    gs = og.boundary_g(lambda X, Y, nx, ny: np.cos(2 * X) * nx + np.sin(3 * Y) * ny)
    b = og.rhs(f, gs)
    ud = methods.direct_solve(og, og.assemble_L(), osys.u_L, b)
    uo, info = methods.algorithm3(osys, b, tol=1e-12)
    lg.factor(tol=1e-12)
    u = zeros(og.r)
    rep = lg.solve(dev(f), u, g=dev(gs))[0]
    assert rep["converged"] == 1
    assert rel(host(u), ud) < 1e-10
    assert rel(host(u), uo) < 1e-10
    assert abs(rep["iterations"] - info["iterations"]) <= 2, (rep, info["iterations"])
