"""CPU checks of the C-ABI library: it loads, exports every symbol that
include/smpm.h declares, rejects bad arguments, and its host factor step
(Sec. 1.2 - 2, computed in C++ with its own GLL nodes, eigen-solver and LU)
matches the oracle.  No GPU is needed: only host entry points are called."""
import os
import re

import numpy as np
import pytest

from paper_1601_03432_gb300 import _binding as B
from oracle.smpm import SMPMGrid, OPPOSITE
from oracle.schur import SchurSystem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1601_03432_gb300.build import build
    build()


def test_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "smpm.h")).read()
    declared = set(re.findall(r"^\s*(?:smpm_status|void|const char\*)\s+(\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations parsed"
    assert declared == set(B.EXPORTS)
    L = B.lib()
    for name in declared:
        assert hasattr(L, name), name


def test_bad_arguments():
    import ctypes
    h = ctypes.c_void_p()
    assert B.lib().smpm_setup(0, 2, 5, 1.0, 1.0, ctypes.byref(h)) == B.SMPM_EINVAL
    assert B.lib().smpm_setup(2, 2, 1, 1.0, 1.0, ctypes.byref(h)) == B.SMPM_EINVAL
    assert B.lib().smpm_setup(2, 2, 33, 1.0, 1.0, ctypes.byref(h)) == B.SMPM_EINVAL
    assert B.lib().smpm_setup(2, 2, 5, -1.0, 1.0, ctypes.byref(h)) == B.SMPM_EINVAL
    g = B.Grid(1, 1, 5)
    with pytest.raises(B.SmpmError) as ei:
        g.factor_host_only()
    assert ei.value.status == B.SMPM_ENOINTERFACE
    g2 = B.Grid(2, 2, 5)
    f = np.zeros(g2.r)
    st = B.lib().schur_solve(g2.h, f.ctypes.data, None, 0.0, 1, f.ctypes.data, None, None)
    assert st == B.SMPM_ESTATE              # no factor yet (nothing is read)
    with pytest.raises(B.SmpmError) as ei:
        g2.solve_host(f, f)
    assert ei.value.status == B.SMPM_ESTATE



def test_coarse_step_beyond_host_memory_is_refused_before_any_work():
    """A 4096 x 4096 grid has d = 33,546,240 interfaces: its dense coarse
    matrices (3 d^2 doubles at least) exceed any host, and the factor step says
    so with ENOMEM at once instead of allocating the element factors first."""
    import time
    g = B.Grid(4096, 4096, 2)
    assert g.d == 2 * 4096 * 4095
    t0 = time.perf_counter()
    with pytest.raises(B.SmpmError) as ei:
        g.factor_host_only()
    assert ei.value.status == B.SMPM_ENOMEM
    assert "coarse" in str(ei.value)
    with pytest.raises(B.SmpmError) as ei:
        B.factor_many([B.Grid(3, 2, 4), g])
    assert ei.value.status == B.SMPM_ENOMEM
    assert time.perf_counter() - t0 < 5.0


class _FakeCudaTensor:
    """Just enough of a CUDA tensor for the binding's argument checks.  Its
    pointer is null: every case below is refused before the library call,
    and the library would refuse a null vector with EINVAL anyway."""
    is_cuda = True

    def __init__(self, n, dtype="torch.float64", contiguous=True):
        self.n, self.dtype, self.contiguous = n, dtype, contiguous

    def is_contiguous(self):
        return self.contiguous

    def numel(self):
        return self.n

    def data_ptr(self):
        return 0


def test_binding_refuses_short_host_or_mistyped_buffers():
    """The C ABI takes vector lengths from the handle, so the binding checks
    every buffer's length, dtype, device and layout before the call."""
    import torch
    g = B.Grid(3, 2, 5)
    T = _FakeCudaTensor
    with pytest.raises(TypeError):
        g.solve(torch.zeros(g.r, dtype=torch.float64), T(g.r))           # host tensor for a device entry
    with pytest.raises(TypeError):
        g.solve(np.zeros(g.r), T(g.r))                                    # NumPy array for a device entry
    with pytest.raises(ValueError):
        g.solve(T(g.r - 1), T(g.r))                                       # f one entry short
    with pytest.raises(ValueError):
        g.solve(T(3 * g.r), T(3 * g.r - 1), nrhs=3)                      # u short for 3 right-hand sides
    with pytest.raises(ValueError):
        g.solve(T(g.r), T(g.r), g=T(g.kp - 1))                            # g short
    with pytest.raises(TypeError):
        g.solve(T(g.r, "torch.float32"), T(g.r))                          # FP32 into an FP64 entry
    with pytest.raises(TypeError):
        g.solve(T(g.r, contiguous=False), T(g.r))
    with pytest.raises(TypeError):
        g.apply_schur32(T(g.kp), T(g.kp, "torch.float32"))                # FP64 into the FP32 operator
    with pytest.raises(ValueError):
        g.schur_rhs(T(g.kp), T(g.kp))                                     # b has r entries, not kp
    with pytest.raises(ValueError):
        g.recover(T(g.r), T(g.kp - 1), T(g.r))
    with pytest.raises(ValueError):
        g.null_vectors(None, None, T(g.d - 1))
    with pytest.raises(ValueError):
        g.solve_adjoint(T(g.r), T(g.r - 1))
    with pytest.raises(ValueError):
        g.solve_host(np.zeros(g.r), np.zeros(g.r - 1))
    with pytest.raises(TypeError):
        g.solve_host(np.zeros(g.r, dtype=np.float32), np.zeros(g.r))


# graded grids (Sec. 1.2): column edges, row edges
GRADED_A = ([0.0, 0.2, 0.5, 1.0, 1.3], [0.0, 0.35, 0.5, 1.1])
GRADED_B = ([0.0, 0.3, 0.45, 1.0], [0.0, 0.5, 1.0, 1.5])     # rows uniform, columns graded
GRIDS = [(2, 2, 6, 1.0, 1.0), (3, 2, 5, 1.5, 0.75), (4, 3, 7, 1.0, 2.0), (5, 4, 4, 1.0, 1.0),
         (4, 3, 6, 0, 0) + GRADED_A, (3, 3, 5, 0, 0) + GRADED_B]


def _grid_ids(p):
    return "x".join(map(str, p[:3])) + ("g" if len(p) > 5 else "")


def _make(p, flags=0):
    mx, my, n, Lx, Ly = p[:5]
    xs, ys = p[5:] if len(p) > 5 else (None, None)
    og = SMPMGrid(mx, my, n, Lx, Ly, xs=xs, ys=ys)
    osys = SchurSystem(og)
    lg = B.Grid(mx, my, n, Lx, Ly, xs=xs, ys=ys)
    lg.factor_host_only(flags=flags)
    return og, osys, lg


@pytest.fixture(scope="module", params=GRIDS, ids=_grid_ids)
def pair(request):
    return _make(request.param)


def test_sizes_and_coords(pair):
    og, osys, lg = pair
    assert (lg.r, lg.kp, lg.d, lg.k) == (og.r, og.kp, og.d, og.k)
    x, y = lg.node_coords()
    ox, oy = og.coords()
    np.testing.assert_allclose(x, ox, atol=1e-14)
    np.testing.assert_allclose(y, oy, atol=1e-14)
    np.testing.assert_allclose(lg.node_mass(), og.mass(), rtol=1e-13)


def test_gll_and_D(pair):
    og, osys, lg = pair
    np.testing.assert_allclose(lg.host_factor("x1d"), og.x1d, atol=1e-15)
    np.testing.assert_allclose(lg.host_factor("w1d"), og.w1d, rtol=1e-13)
    n = og.n
    np.testing.assert_allclose(lg.host_factor("D").reshape(n, n), og.D, atol=1e-12 * n * n)


def test_T_blocks_are_S_entries(pair):
    """T_e[(F,t),(G,s)] = S[slot (nbr(e,F), opp F, t), slot (e,G,s)]."""
    og, osys, lg = pair
    n, M = og.n, 4 * og.n
    T = lg.host_factor("T").reshape(og.nel, M, M)
    Sd = osys.S.toarray()
    scale = np.abs(Sd).max()
    for e in range(og.nel):
        for F in range(4):
            e2 = og.neighbour(e, F)
            for G in range(4):
                for t in range(n):
                    for s in range(n):
                        val = T[e, F * n + t, G * n + s]
                        if e2 < 0 or og.neighbour(e, G) < 0:
                            assert val == 0.0
                            continue
                        ref = Sd[og.slot_of[(e2, OPPOSITE[F], t)], og.slot_of[(e, G, s)]]
                        assert abs(val - ref) <= 1e-11 * scale


def test_block_jacobi_reduced_form(pair):
    """M_b^-1 through G = (I - X Y)^-1: a = G (p - X q), b = q - T_e a."""
    og, osys, lg = pair
    n, M = og.n, 4 * og.n
    T = lg.host_factor("T").reshape(og.nel, M, M)
    G = lg.host_factor("G").reshape(-1, M, M)
    X = lg.host_factor("X").reshape(-1, 4, n, n)
    black = lg.host_factor("black").astype(int)
    assert list(black) == osys.black
    v = np.random.default_rng(4).standard_normal(og.k)
    ref = osys.apply_Minv(v)
    vp = og.to_padded(v)
    out = np.zeros(og.kp)
    for ib, e in enumerate(black):
        p = vp[e * M:(e + 1) * M].copy()
        q = np.zeros(M)
        for F in range(4):
            e2 = og.neighbour(e, F)
            if e2 >= 0:
                q[F * n:(F + 1) * n] = vp[e2 * M + OPPOSITE[F] * n: e2 * M + OPPOSITE[F] * n + n]
        Xq = np.concatenate([X[ib, F] @ q[F * n:(F + 1) * n] for F in range(4)])
        a = G[ib] @ (p - Xq)
        b = q - T[e] @ a
        out[e * M:(e + 1) * M] = a
        for F in range(4):
            e2 = og.neighbour(e, F)
            if e2 >= 0:
                out[e2 * M + OPPOSITE[F] * n: e2 * M + OPPOSITE[F] * n + n] = b[F * n:(F + 1) * n]
    np.testing.assert_allclose(og.from_padded(out), ref, atol=1e-10 * np.abs(ref).max())


def test_coarse_objects(pair):
    og, osys, lg = pair
    d = og.d
    C = lg.coarse_matrix()
    np.testing.assert_allclose(C, osys.C, atol=1e-11 * np.abs(osys.C).max())
    # deflation weights (1 on uniform grids) and B 1 = Z c0
    zw = lg.host_factor("zw").reshape(og.nel, 4)
    w = np.array([zw[e, F] for (e, F, t) in og.slots])
    np.testing.assert_allclose(w, osys.zweights, rtol=1e-14)
    np.testing.assert_allclose(og.from_padded(lg.host_factor("B1")), osys.B1, rtol=1e-14)
    c0 = lg.host_factor("c0")
    assert abs(abs(c0 @ osys.c0) / (np.linalg.norm(c0) * np.linalg.norm(osys.c0)) - 1) < 1e-13
    uC = lg.host_factor("uC")
    assert abs(abs(uC @ osys.u_C) - 1) < 1e-11
    H = lg.host_factor("H").reshape(d, d)
    r = np.random.default_rng(5).standard_normal(d)
    np.testing.assert_allclose(H @ r, osys.coarse_solve(r), atol=1e-9 * np.abs(osys.coarse_solve(r)).max())


def test_null_vectors(pair):
    """u_S and u_L to round-off: a direction error leaves an inconsistent
    component in b_S that stalls GMRES near the tolerance."""
    og, osys, lg = pair
    uS = og.from_padded(lg.host_factor("uS"))
    uS *= np.sign(uS @ osys.u_S)
    assert np.linalg.norm(uS - osys.u_S) < 1e-12
    assert np.linalg.norm(osys.S.T @ uS) < 1e-13 * abs(osys.S).max() * np.sqrt(og.k)
    uL = lg.host_factor("uL")
    uL *= np.sign(uL @ osys.u_L)
    assert np.linalg.norm(uL - osys.u_L) < 1e-12
    np.testing.assert_allclose(lg.host_factor("what").sum(), 1.0, rtol=1e-14)


# ---------------------------------------------------- transposed system
@pytest.fixture(scope="module", params=GRIDS[1:3] + GRIDS[4:5], ids=_grid_ids)
def apair(request):
    return _make(request.param, flags=B.FLAG_ADJOINT)


def _phi(og):
    """The slot swap Phi on compact slots: (e, F, t) <-> (nbr(e, F), opp F, t)."""
    p = np.empty(og.k, dtype=np.int64)
    for i, (e, F, t) in enumerate(og.slots):
        p[i] = og.slot_of[(og.neighbour(e, F), OPPOSITE[F], t)]
    return p


def test_adjoint_T_is_transpose(apair):
    og, osys, lg = apair
    M = 4 * og.n
    T = lg.host_factor("T").reshape(og.nel, M, M)
    Ta = lg.host_factor("Ta").reshape(og.nel, M, M)
    assert np.array_equal(Ta, T.transpose(0, 2, 1))
    # I + push(T~) is Phi S^T Phi
    phi = _phi(og)
    v = np.random.default_rng(8).standard_normal(og.k)
    vp = og.to_padded(v)
    yp = vp.copy()
    n = og.n
    for e in range(og.nel):
        z = Ta[e] @ vp[e * M:(e + 1) * M]
        for F in range(4):
            e2 = og.neighbour(e, F)
            if e2 >= 0:
                yp[e2 * M + OPPOSITE[F] * n: e2 * M + OPPOSITE[F] * n + n] += z[F * n:(F + 1) * n]
    ref = (osys.S.T @ v[phi])[phi]
    np.testing.assert_allclose(og.from_padded(yp), ref, atol=1e-11 * np.abs(ref).max())


def test_adjoint_block_jacobi_is_transposed(apair):
    """The reduced form with (T~, G~, X~) applies Phi M^-T Phi."""
    og, osys, lg = apair
    n, M = og.n, 4 * og.n
    T = lg.host_factor("Ta").reshape(og.nel, M, M)
    G = lg.host_factor("Ga").reshape(-1, M, M)
    X = lg.host_factor("Xa").reshape(-1, 4, n, n)
    black = lg.host_factor("black").astype(int)
    phi = _phi(og)
    v = np.random.default_rng(4).standard_normal(og.k)
    ref = osys.apply_MinvT(v[phi])[phi]
    vp = og.to_padded(v)
    out = np.zeros(og.kp)
    for ib, e in enumerate(black):
        p = vp[e * M:(e + 1) * M].copy()
        q = np.zeros(M)
        for F in range(4):
            e2 = og.neighbour(e, F)
            if e2 >= 0:
                q[F * n:(F + 1) * n] = vp[e2 * M + OPPOSITE[F] * n: e2 * M + OPPOSITE[F] * n + n]
        Xq = np.concatenate([X[ib, F] @ q[F * n:(F + 1) * n] for F in range(4)])
        a = G[ib] @ (p - Xq)
        b = q - T[e] @ a
        out[e * M:(e + 1) * M] = a
        for F in range(4):
            e2 = og.neighbour(e, F)
            if e2 >= 0:
                out[e2 * M + OPPOSITE[F] * n: e2 * M + OPPOSITE[F] * n + n] = b[F * n:(F + 1) * n]
    np.testing.assert_allclose(og.from_padded(out), ref, atol=1e-10 * np.abs(ref).max())


def test_adjoint_coarse_and_null_vectors(apair):
    from oracle.adjoint import AdjointDeflation
    og, osys, lg = apair
    d = og.d
    Ha = lg.host_factor("Ha").reshape(d, d)
    r = np.random.default_rng(6).standard_normal(d)
    ref = AdjointDeflation(osys).coarse_solve(r)
    np.testing.assert_allclose(Ha @ r, ref, atol=1e-9 * np.abs(ref).max())
    # left null vector of Phi S^T Phi: Phi B1 (= B1 where B1 is constant on
    # every interface)
    phi = _phi(og)
    uSa = og.from_padded(lg.host_factor("uSa"))
    ref = (osys.B1 / np.linalg.norm(osys.B1))[phi]
    assert np.linalg.norm(uSa * np.sign(uSa @ ref) - ref) < 1e-14
    assert np.linalg.norm(osys.S @ uSa[phi]) < 1e-12 * abs(osys.S).max()


def test_transposed_fast_diagonalisation(apair):
    og, osys, lg = apair
    n = og.n
    fd, fdT = lg.host_factor("fdx"), lg.host_factor("fdxT")
    fds = 2 * n * n + n
    for cls in range(len(fd) // fds):
        V, Vi, lam = (fd[cls * fds:cls * fds + n * n].reshape(n, n),
                      fd[cls * fds + n * n:cls * fds + 2 * n * n].reshape(n, n), fd[cls * fds + 2 * n * n:(cls + 1) * fds])
        W, Wi, lamT = (fdT[cls * fds:cls * fds + n * n].reshape(n, n),
                       fdT[cls * fds + n * n:cls * fds + 2 * n * n].reshape(n, n),
                       fdT[cls * fds + 2 * n * n:(cls + 1) * fds])
        K = V @ np.diag(lam) @ Vi
        np.testing.assert_allclose(W @ np.diag(lamT) @ Wi, K.T, atol=1e-10 * np.abs(K).max())


def test_coarse_inverse_accuracy_on_elongated_grid():
    """The regularised coarse inverse H solves C y = r' (r' = r projected
    out of u_C) to near round-off also where the grid is elongated and C is
    poorly conditioned (aspect ratio 6 here): GMRES stops relative to the
    deflated right-hand side, so the coarse solve's error is a floor for
    the attainable residual."""
    lg = B.Grid(4, 25, 14)
    lg.factor_host_only()
    d = lg.d
    H = lg.host_factor("H").reshape(d, d)
    C = lg.coarse_matrix()
    uC = lg.host_factor("uC")
    r = np.random.default_rng(3).standard_normal(d)
    r -= uC * (uC @ r)
    y = H @ r
    assert np.linalg.norm(C @ y - r) <= 1e-12 * np.linalg.norm(r)


@pytest.mark.parametrize("mx,my,n", [(5, 4, 6), (8, 7, 5)])
def test_factors_are_identical_within_a_class(mx, my, n):
    """The host null-vector solve reads one representative per class: T_e of
    elements with the same face-type mask, G_b and X_b of black blocks with
    the same own and neighbour masks.  That is exact only if the stored
    per-element copies are bitwise equal within a class."""
    g = B.Grid(mx, my, n)
    g.factor_host_only()
    M = 4 * n
    T = g.host_factor("T").reshape(mx * my, M, M)
    Gb = g.host_factor("G").reshape(-1, M, M)
    Xb = g.host_factor("X").reshape(-1, 4 * n * n)
    black = g.host_factor("black").astype(int)

    def nb(e, F):
        ix, iy = e % mx, e // mx
        return [e - 1 if ix > 0 else -1, e + 1 if ix < mx - 1 else -1,
                e - mx if iy > 0 else -1, e + mx if iy < my - 1 else -1][F]

    def mask(e):
        return sum(1 << F for F in range(4) if nb(e, F) >= 0)

    first = {}
    for e in range(mx * my):
        r = first.setdefault(mask(e), e)
        assert np.array_equal(T[e], T[r])
    firstb = {}
    for ib, e in enumerate(black):
        key = (mask(e),) + tuple(mask(nb(e, F)) if nb(e, F) >= 0 else 0 for F in range(4))
        r = firstb.setdefault(key, ib)
        assert np.array_equal(Gb[ib], Gb[r]) and np.array_equal(Xb[ib], Xb[r])
    assert len(first) <= 9


def test_graded_setup_rejects_bad_edges():
    """smpm_setup_graded: edges must be finite and strictly increasing, one
    more than the element count in each direction."""
    with pytest.raises(B.SmpmError) as ei:
        B.Grid(3, 2, 4, xs=[0.0, 0.5, 0.5, 1.0], ys=[0.0, 0.3, 1.0])
    assert ei.value.status == B.SMPM_EINVAL
    with pytest.raises(B.SmpmError):
        B.Grid(3, 2, 4, xs=[0.0, 0.5, np.nan, 1.0], ys=[0.0, 0.3, 1.0])
    with pytest.raises(B.SmpmError):
        B.Grid(3, 2, 4, xs=[0.0, 0.5, 0.7, 1.0], ys=[0.0, 1.0, 0.3])
    with pytest.raises(ValueError):
        B.Grid(3, 2, 4, xs=[0.0, 0.5, 1.0], ys=[0.0, 0.3, 1.0])
    g = B.Grid(3, 2, 4, xs=[-1.0, 0.5, 0.7, 1.0], ys=[2.0, 2.3, 3.0])
    x, y = g.node_coords()
    assert x.min() == -1.0 and x.max() == 1.0 and y.min() == 2.0 and y.max() == 3.0
    assert abs(g.node_mass().sum() - 2.0 * 1.0) < 1e-13


def test_partition_rejects_bad_tiles():
    g = B.Grid(4, 3, 4)
    for px, py, rank in ((0, 1, 0), (5, 1, 0), (2, 4, 0), (2, 2, 4), (2, 2, -1)):
        with pytest.raises(B.SmpmError) as ei:
            g.partition_tile(px, py, rank)
        assert ei.value.status == B.SMPM_EINVAL
    t = g.partition_tile(2, 3, 5)
    assert (t["ix0"], t["ix1"], t["iy0"], t["iy1"]) == (2, 4, 2, 3)
    assert t["peers"] == [4, -1, 3, -1] and t["halo"] == [4, 0, 8, 0]
