"""Schur complement, null vectors, block-Jacobi and deflation operators.

Sec. 1.3 (Eq. blocksystem, operator_decomp, schur_complement_system):
    S = I + B A^-1 E  (k x k),   b_S = B A^-1 f,   u = A^-1 (f - E v).
Sec. 1.4 (Eq. regularize_poisson, regularize_schur): L and S have one-
dimensional left null spaces spanned by the unit vectors u_L and u_S; the
right-hand sides are projected out of them.
Sec. 2 (Fig. 2): block-Jacobi M with one block per element of one checkerboard
colour, holding its interfaces on both sides; deflation with the interface
indicator vectors Z, C = Z^T S Z (Eq. after the definition of z_j), and the
projections P = I - S Z C^-1 Z^T (Eq. projection1), Q = I - Z C^-1 Z^T S
(Eq. projection2).  C inherits the rank deficiency of S and every application
of C^-1 is regularised with the left null vector u_C of C.

Readings of passages the paper leaves open:
* The right null vector of L is the constant vector (Sec. 1.4), so B 1 is a
  right null vector of S (A 1 + E B 1 = L 1 = 0 gives B A^-1 E (B 1) = -B 1).
  B 1 = -tau_F p_F of the receiving face.  Where both sides of every interface
  carry the same tau_F p_F (uniform grids), B 1 = Z c0 and C c0 = 0.
* "C \\ r" for the singular C is read as: project r out of u_C, then take the
  solution y of C y = r' with c0^T y = 0 (a bordered solve).  Any other choice
  changes the Schur solution only by a multiple of B 1, i.e. u only by a
  constant, which the zero-mean normalisation removes.
* On a graded grid where some interface has different h_perp on its two sides,
  B 1 is not in the range of Z; C is then nonsingular and C \\ r is the plain
  solve (no u_C, no border).
* The black checkerboard colour is i_x + i_y even.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .smpm import W, E, S, N, OPPOSITE


class SchurSystem:
    """All operators of Algorithms 1-3 for one grid (FP64, plain)."""

    def __init__(self, grid, seed=12345, deflation="weighted"):
        """deflation: "weighted" (z_j = B 1 on interface j's slots over the mean
        of its two sides, the indicator on a uniform grid) or "indicator" (the
        0/1 vectors of Sec. 2 on any grid)."""
        if deflation not in ("weighted", "indicator"):
            raise ValueError("deflation must be 'weighted' or 'indicator'")
        self.deflation = deflation
        if grid.nel < 2:
            raise ValueError("the Schur method needs at least one interface (m_x m_y >= 2)")
        self.grid = grid
        self.rng = np.random.default_rng(seed)
        g = grid
        # A is block diagonal (Sec. 1.3); one dense LU per element.  Elements
        # with the same A_e matrix share the factorisation (identical input,
        # identical output).
        self._lu_cache = {}
        self.A_lu = []
        for e in range(g.nel):
            key = tuple(g.neighbour(e, F) >= 0 for F in (W, E, S, N)) + tuple(g.h_of(e))
            if key not in self._lu_cache:
                self._lu_cache[key] = sla.lu_factor(g.element_A(e))
            self.A_lu.append(self._lu_cache[key])
        self.B = g.assemble_B()
        self.E = g.assemble_E()
        self.AinvE = self._assemble_AinvE()
        # S = I + B A^-1 E (Eq. schur_complement_system)
        self.S = (sp.identity(g.k, format="csr") + self.B @ self.AinvE).tocsr()
        self.B1 = self.B @ np.ones(g.r)
        self._build_blocks()
        self._build_deflation()
        self.u_S = self.left_null_S()
        self.u_L = self.left_null_L_from_uS()

    # ---------------------------------------------------------- element solves
    def A_solve(self, b):
        """A^-1 b, element by element (A is block diagonal, Sec. 1.3)."""
        g = self.grid
        out = np.empty(g.r)
        for e in range(g.nel):
            sl = slice(e * g.nn, (e + 1) * g.nn)
            out[sl] = sla.lu_solve(self.A_lu[e], b[sl])
        return out

    def AT_solve(self, b):
        """A^-T b, element by element."""
        g = self.grid
        out = np.empty(g.r)
        for e in range(g.nel):
            sl = slice(e * g.nn, (e + 1) * g.nn)
            out[sl] = sla.lu_solve(self.A_lu[e], b[sl], trans=1)
        return out

    def _assemble_AinvE(self):
        """A^-1 E as a sparse r x k matrix: column (e,F,t) is A_e^-1 applied to
        the unit vector at the face node of slot (e,F,t)."""
        g = self.grid
        rows, cols, vals = [], [], []
        per_elem = {}
        for i, (e, F, t) in enumerate(g.slots):
            per_elem.setdefault(e, []).append((i, F, t))
        for e in range(g.nel):
            lst = per_elem.get(e, [])
            if not lst:
                continue
            rhs = np.zeros((g.nn, len(lst)))
            for c, (_, F, t) in enumerate(lst):
                a, b = g.face_node(F, t)
                rhs[b * g.n + a, c] = 1.0
            sol = sla.lu_solve(self.A_lu[e], rhs)
            rr, cc = np.meshgrid(np.arange(g.nn), [i for (i, _, _) in lst], indexing="ij")
            rows.append(e * g.nn + rr.ravel()); cols.append(cc.ravel()); vals.append(sol.ravel())
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(g.r, g.k)).tocsr()

    # ------------------------------------------------------------- operators
    def apply_S(self, v):
        """S v = v + B A^-1 E v (matrix-free form of Eq. schur_complement_system)."""
        return v + self.B @ self.A_solve(self.E @ v)

    def apply_ST(self, v):
        """S^T v = v + E^T A^-T B^T v."""
        return v + self.E.T @ self.AT_solve(self.B.T @ v)

    def schur_rhs(self, b):
        """b_S = B A^-1 b (right-hand side of Eq. schur_complement_system)."""
        return self.B @ self.A_solve(b)

    def recover(self, b, x):
        """u = A^-1 (b - E x) (back-substitution after Eq. schur_complement_system)."""
        return self.A_solve(b - self.E @ x)

    # ----------------------------------------------------------- null vectors
    def left_null_S(self):
        """Unit u_S with u_S^T S = 0 (Sec. 1.4), from the nonsingular bordered
        system [[S^T, B1], [a^T, 0]] [y; eta] = [0; 1] with a seeded random a
        (multiplying the first block row by (B1)^T shows eta = 0)."""
        g = self.grid
        a = self.rng.standard_normal(g.k)
        K = sp.bmat([[self.S.T, sp.csr_matrix(self.B1[:, None])],
                     [sp.csr_matrix(a[None, :]), None]], format="csc")
        rhs = np.zeros(g.k + 1)
        rhs[-1] = 1.0
        y = spla.splu(K).solve(rhs)[: g.k]
        y /= np.linalg.norm(y)
        return _fix_sign(y)

    def left_null_L_from_uS(self):
        """u_L from u_S: u_L proportional to -A^-T B^T u_S, since then
        u_L^T L = -u_S^T B A^-1 (A + E B) = -u_S^T S B = 0."""
        y = -self.AT_solve(self.B.T @ self.u_S)
        y /= np.linalg.norm(y)
        return _fix_sign(y)

    # ---------------------------------------------------------- block Jacobi
    def _build_blocks(self):
        """Checkerboard blocks of M (Sec. 2, Fig. 2): for every black element
        (i_x + i_y even) its own interface slots followed by the neighbours'
        slots facing it; these blocks partition Gamma.  M_b = S[block, block]."""
        g = self.grid
        self.black = [e for e in range(g.nel) if sum(g.element_ij(e)) % 2 == 0]
        self.blocks = []
        self.block_lu = []
        for e in self.black:
            own, facing = [], []
            for F in (W, E, S, N):
                e2 = g.neighbour(e, F)
                if e2 < 0:
                    continue
                for t in range(g.n):
                    own.append(g.slot_of[(e, F, t)])
                    facing.append(g.slot_of[(e2, OPPOSITE[F], t)])
            idx = np.array(own + facing, dtype=np.int64)
            Mb = self.S[idx][:, idx].toarray()
            self.blocks.append(idx)
            self.block_lu.append(sla.lu_factor(Mb))
        covered = np.sort(np.concatenate(self.blocks)) if self.blocks else np.array([], int)
        if not np.array_equal(covered, np.arange(g.k)):
            raise AssertionError("block-Jacobi blocks do not partition Gamma")

    def apply_Minv(self, v):
        """M^-1 v, block by block."""
        out = np.zeros_like(v)
        for idx, lu in zip(self.blocks, self.block_lu):
            out[idx] = sla.lu_solve(lu, v[idx])
        return out

    def apply_MinvT(self, v):
        out = np.zeros_like(v)
        for idx, lu in zip(self.blocks, self.block_lu):
            out[idx] = sla.lu_solve(lu, v[idx], trans=1)
        return out

    # -------------------------------------------------------------- deflation
    def _build_deflation(self):
        """Z (k x d): z_j is 1 on the 2n slots of interface j (both sides) and 0
        elsewhere; C = Z^T S Z (Sec. 2).  Graded-grid reading: B 1 takes the
        value -tau_F p_F of each side, which differs across an interface of
        unequal sizes, so with 0/1 vectors B 1 leaves the coarse space (C is
        then nonsingular) and deflated GMRES stagnates on strongly graded grids.
        The weighted z_j is B 1 restricted to interface j divided by beta_j, the
        mean of its two sides; B 1 = Z beta again, and on a uniform grid every
        weight is exactly 1."""
        g = self.grid
        cols = np.array([g.iface_of[(e, F)] for (e, F, t) in g.slots])
        beta = np.empty(g.d)                     # mean of the two sides' values
        for j, (e, F) in enumerate(g.interfaces):
            e2 = g.neighbour(e, F)
            beta[j] = 0.5 * (self.B1[g.slot_of[(e, F, 0)]] + self.B1[g.slot_of[(e2, OPPOSITE[F], 0)]])
        w = self.B1 / beta[cols] if self.deflation == "weighted" else np.ones(g.k)
        self.zweights = w
        self.Z = sp.csr_matrix((w, (np.arange(g.k), cols)), shape=(g.k, g.d))
        self.C = (self.Z.T @ (self.S @ self.Z)).toarray()
        # right null vector of C: B 1 = Z c0 when B 1 is in the range of Z
        c0 = beta
        self.coarse_singular = bool(np.allclose(self.Z @ c0, self.B1, rtol=1e-12,
                                                atol=1e-12 * np.abs(self.B1).max()))
        d = g.d
        if not self.coarse_singular:
            self.c0, self.u_C = None, None
            self.C_lu = sla.lu_factor(self.C)
            return
        self.c0 = c0
        K = np.zeros((d + 1, d + 1))
        K[:d, :d] = self.C
        K[:d, d] = self.c0
        K[d, :d] = self.c0
        self.K_lu = sla.lu_factor(K)
        # u_C: unit left null vector of C, from K^T [y; eta] = [0; 1]
        rhs = np.zeros(d + 1)
        rhs[d] = 1.0
        y = sla.lu_solve(self.K_lu, rhs, trans=1)[:d]
        y /= np.linalg.norm(y)
        self.u_C = _fix_sign(y)

    def coarse_solve(self, r):
        """C\\ r regularised (Sec. 2): y with C y = r - u_C (u_C^T r), c0^T y = 0
        (a plain solve when C is nonsingular)."""
        if not self.coarse_singular:
            return sla.lu_solve(self.C_lu, r)
        d = self.grid.d
        rr = r - self.u_C * (self.u_C @ r)
        return sla.lu_solve(self.K_lu, np.concatenate([rr, [0.0]]))[:d]

    def apply_P(self, y):
        """P y = y - S Z C\\ Z^T y (Eq. projection1)."""
        return y - self.apply_S(self.Z @ self.coarse_solve(self.Z.T @ y))

    def apply_Q(self, x):
        """Q x = x - Z C\\ Z^T S x (Eq. projection2)."""
        return x - self.Z @ self.coarse_solve(self.Z.T @ self.apply_S(x))


def _fix_sign(v):
    """Null vectors are defined up to sign; make the largest-magnitude entry positive."""
    i = int(np.argmax(np.abs(v)))
    return v if v[i] >= 0 else -v
