"""GPU parity of the adjoint solve (schur_solve_adjoint) and its autograd
binding against the oracle's adjoint, the inner-product identity of the
forward and adjoint GPU solves, and central finite differences of the
quadratic loss ||u - u_t||^2 on the 48 x 48, n = 16 grid.

Tolerances: dl/df, dl/dg to a relative L2 error of 1e-10 against the oracle
(FP64, tol 1e-12), iteration counts within one of the oracle's Algorithm 3 on
S^T; the identity to 1e-10; finite differences as stated in the config-5
test (the quotient of a quadratic loss has no truncation error, only the two
solves' errors divided by 2h)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1601_03432_gb300 import Grid, inputs
from paper_1601_03432_gb300 import _binding as B
from paper_1601_03432_gb300.autograd import schur_solve
from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import adjoint

GRIDS = [(2, 2, 8, 1.0, 1.0), (3, 2, 5, 1.5, 0.75), (5, 4, 7, 1.0, 1.0), (1, 3, 4, 1.0, 2.0), (9, 7, 5, 1.0, 1.0)]


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


@pytest.fixture(scope="module", params=GRIDS, ids=lambda p: "x".join(map(str, p[:3])))
def pair(request, built):
    mx, my, n, Lx, Ly = request.param
    og = SMPMGrid(mx, my, n, Lx, Ly)
    osys = SchurSystem(og)
    lg = Grid(mx, my, n, Lx, Ly)
    return og, osys, lg


@pytest.mark.parametrize("flags", [0, 1, 2, 8], ids=["smem", "global", "stream", "warps"])
@pytest.mark.parametrize("precond", [0, 1, 2])
def test_adjoint_matches_oracle(pair, precond, flags):
    og, osys, lg = pair
    if og.d < 2 and precond > 0:
        pytest.skip("single interface")
    gbar = inputs.white_noise(og.r, 31) + 0.25          # non-zero sum exercises N^T
    db_ref = adjoint.adjoint_direct(og, og.assemble_L(), osys.u_L, gbar)
    df_ref, dg_ref = adjoint.grad_f_g(og, db_ref)
    lg.factor(precond=precond, tol=1e-12, flags=flags | B.FLAG_ADJOINT)
    gf = torch.zeros(og.r, dtype=torch.float64, device="cuda")
    gg = torch.full((og.kp,), 7.0, dtype=torch.float64, device="cuda")
    rep = lg.solve_adjoint(dev(gbar), gf, gg)[0]
    assert rep["converged"] == 1
    assert rel(host(gf), df_ref) < 1e-10, rep
    assert rel(host(gg), dg_ref) < 1e-10
    if precond == 2:
        _, info = adjoint.algorithm3_adjoint(osys, gbar, tol=1e-12, restart=50)
        assert abs(rep["iterations"] - info["iterations"]) <= 1, (rep, info["iterations"])
    assert rep["schur_relres"] < 1e-10


def test_adjoint_needs_flag(built):
    lg = Grid(3, 3, 5)
    lg.factor()
    x = torch.zeros(lg.r, dtype=torch.float64, device="cuda")
    with pytest.raises(B.SmpmError) as ei:
        lg.solve_adjoint(x, x)
    assert ei.value.status == B.SMPM_ESTATE


def test_adjoint_of_mixed_precision_handle(built):
    """A handle factored with precision 1 still runs the adjoint in FP64."""
    og = SMPMGrid(4, 4, 6)
    osys = SchurSystem(og)
    lg = Grid(4, 4, 6)
    lg.factor(precision=1, tol=1e-12, flags=B.FLAG_ADJOINT)
    gbar = inputs.white_noise(og.r, 3)
    gf = torch.zeros(og.r, dtype=torch.float64, device="cuda")
    lg.solve_adjoint(dev(gbar), gf)
    ref = adjoint.adjoint_direct(og, og.assemble_L(), osys.u_L, gbar)
    assert rel(host(gf), ref) < 1e-10


def test_medium_grid_matches_oracle_algorithm3(built):
    """8 x 8 elements, n = 16 (the config-5 polynomial order on a grid the
    oracle's Algorithm 3 finishes in seconds)."""
    og = SMPMGrid(8, 8, 16)
    osys = SchurSystem(og)
    lg = Grid(8, 8, 16)
    lg.factor(tol=1e-11, flags=B.FLAG_ADJOINT)
    x, y = og.coords()
    ut, _ = inputs.fourier_rhs(x, y, seed=5)
    f, _ = inputs.fourier_rhs(x, y, seed=6)
    u = torch.zeros(og.r, dtype=torch.float64, device="cuda")
    lg.solve(dev(f), u)
    gbar = 2 * (host(u) - ut)
    db_ref, info = adjoint.algorithm3_adjoint(osys, gbar, tol=1e-11, restart=50)
    gf = torch.zeros(og.r, dtype=torch.float64, device="cuda")
    rep = lg.solve_adjoint(dev(gbar), gf)[0]
    assert abs(rep["iterations"] - info["iterations"]) <= 1, (rep, info["iterations"])
    assert rel(host(gf), db_ref) < 1e-9


def test_inner_product_identity(built):
    """<gbar, u(f, g)> = <dl/df, f> + <dl/dg, g> for the GPU forward and
    adjoint solves (u is linear in f and g)."""
    lg = Grid(16, 12, 10, 1.0, 0.75)
    lg.factor(tol=1e-12, flags=B.FLAG_ADJOINT)
    rng = np.random.default_rng(9)
    f, gs, gbar = rng.standard_normal(lg.r), rng.standard_normal(lg.kp), rng.standard_normal(lg.r)
    u = torch.zeros(lg.r, dtype=torch.float64, device="cuda")
    lg.solve(dev(f), u, g=dev(gs))
    gf = torch.zeros(lg.r, dtype=torch.float64, device="cuda")
    gg = torch.zeros(lg.kp, dtype=torch.float64, device="cuda")
    lg.solve_adjoint(dev(gbar), gf, gg)
    lhs = gbar @ host(u)
    rhs = host(gf) @ f + host(gg) @ gs
    assert abs(lhs - rhs) <= 1e-10 * np.linalg.norm(gbar) * np.linalg.norm(host(u)) * 10


def test_autograd_matches_adjoint(built):
    og = SMPMGrid(5, 4, 7)
    osys = SchurSystem(og)
    lg = Grid(5, 4, 7)
    lg.factor(tol=1e-12, flags=B.FLAG_ADJOINT)
    rng = np.random.default_rng(12)
    f = dev(rng.standard_normal((2, og.r))).requires_grad_(True)
    g = dev(rng.standard_normal((2, og.kp))).requires_grad_(True)
    ut = dev(rng.standard_normal((2, og.r)))
    u = schur_solve(lg, f, g, tol=1e-12)
    loss = ((u - ut) ** 2).sum()
    loss.backward()
    Lm = og.assemble_L()
    for k in range(2):
        db = adjoint.adjoint_direct(og, Lm, osys.u_L, 2 * (host(u[k]) - host(ut[k])))
        df, dg = adjoint.grad_f_g(og, db)
        assert rel(host(f.grad[k]), df) < 1e-10
        assert rel(host(g.grad[k]), dg) < 1e-10


@pytest.mark.slow
def test_config5_finite_differences(built):
    """48 x 48 elements, n = 16: loss ||u - u_t||^2 with a seeded smooth u_t;
    dl/df and dl/dg from the autograd backward against central differences on
    64 random directions in (f, g), solver tol 1e-11 (a tighter tolerance
    stagnates in FP64 on this grid).  The loss is quadratic in (f, g), so
    central differences carry no truncation error at any h: the quotient
    differs from the derivative only by the difference of the two solves'
    errors divided by 2h.  At h = 1e-6 that is ~1e-11 |u| / h (bound 5e-5
    relative); at h = 1e-2 it is ~1e-9, which checks the gradient itself."""
    lg = Grid(48, 48, 16)
    tol = 1e-11
    lg.factor(tol=tol, flags=B.FLAG_ADJOINT)
    x, y = lg.node_coords()
    ut = dev(inputs.fourier_rhs(x, y, seed=5)[0])
    f0 = dev(inputs.fourier_rhs(x, y, seed=6)[0])
    g0 = torch.zeros(lg.kp, dtype=torch.float64, device="cuda")
    f = f0.clone().requires_grad_(True)
    g = g0.clone().requires_grad_(True)
    loss = ((schur_solve(lg, f, g, tol=tol) - ut) ** 2).sum()
    loss.backward()
    for h, bound, ndir in ((1e-6, 5e-5, 64), (1e-2, 1e-8, 8)):
        gen = torch.Generator(device="cuda").manual_seed(11)
        worst = 0.0
        with torch.no_grad():
            for k in range(ndir):
                pf = torch.randn(lg.r, dtype=torch.float64, device="cuda", generator=gen)
                pg = torch.randn(lg.kp, dtype=torch.float64, device="cuda", generator=gen)
                lp = ((schur_solve(lg, f0 + h * pf, g0 + h * pg, tol=tol) - ut) ** 2).sum()
                lm = ((schur_solve(lg, f0 - h * pf, g0 - h * pg, tol=tol) - ut) ** 2).sum()
                fd = float((lp - lm) / (2 * h))
                an = float(f.grad @ pf + g.grad @ pg)
                worst = max(worst, abs(fd - an) / max(abs(an), 1e-30))
        assert worst < bound, (h, worst)
