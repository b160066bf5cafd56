"""SMPM discretisation of the 2-D Poisson-Neumann problem (Sec. 1.2 - 1.3).

Conventions fixed here (the paper leaves them open; each is a reading of the
passage cited):

* Elements: an m_y x m_x Cartesian grid on [0, L_x] x [0, L_y] (Sec. 1.2, Sec. 3),
  element e = i_y * m_x + i_x covering [i_x h_x, (i_x+1) h_x] x [i_y h_y, (i_y+1) h_y].
  Graded grids (Sec. 1.2 allows any smooth invertible element map; the
  axis-aligned case is taken): column edges x_0 < ... < x_mx and row edges
  y_0 < ... < y_my, element (i_x, i_y) covering [x_ix, x_ix+1] x [y_iy, y_iy+1],
  so h_x varies by column and h_y by row and neighbours stay conforming.
* Graded readings of Eq. smpm_poisson: tau_F and p_F of a face use the h_perp of
  the element that owns the face (the element whose residual row it is), so the
  two sides of an interface may carry different values; in element e's
  residual the neighbour's trace enters through the same R (e's p_F), and the
  neighbour's gradient is taken with the neighbour's own map.  The jump of R u
  then vanishes for any smooth u, as on a uniform grid.
* Nodes: n x n GLL points per element, node (a, b) at local index b * n + a (the
  x index a runs fastest), global index e * n^2 + b * n + a; r = n^2 m_x m_y.
* Faces: W, E, S, N = 0, 1, 2, 3 with outward normals (-1,0), (1,0), (0,-1),
  (0,1).  Face node t runs along the face in increasing coordinate: W/E face
  node t is (a = 0 / n-1, b = t); S/N face node t is (a = t, b = 0 / n-1).
* Penalty and Robin weight (Eq. smpm_poisson; the paper calls tau_i a
  heuristic and gives no value, and writes the Robin flux R = I + n.grad
  without a length scale while leaving L_x, L_y unstated).  The face terms are
      tau_F [ p_F (u_e - u_e') + n_F.grad u_e - n_F.grad u_e' ]  (interface),
      tau_F n_F.grad u_e                                         (boundary),
  right-hand side f + tau_F g, with
      tau_F = -alpha n (n - 1) / h_perp,   p_F = beta n (n - 1) / h_perp,
  h_perp = h_x on W/E faces and h_y on S/N faces, alpha = 1, beta = 1/4 by
  default.  alpha = 1 makes the face terms equal the GLL-quadrature weak form
  divided by the nodal mass; p_F is the weight of the identity in R relative
  to the normal derivative, expressed in the element's own length scale.
  The literal reading of R = I + n.grad (p_F = 1 on every face, whatever the
  element size) is available with robin_literal=True.
* Interface unknowns (Sec. 1.3): one slot per (element, interface face, face
  node), so each interface carries 2n slots (n on either side) and a corner node
  of an element appears in two slots.  Padded slot index e * 4n + F * n + t;
  the oracle also numbers the k = 2 n d real (interface) slots compactly in the
  same order.
* Interfaces: d = (m_x - 1) m_y + m_x (m_y - 1), numbered row by row: for each
  element row i_y, first the m_x - 1 vertical interfaces (between i_x and
  i_x + 1), then the m_x horizontal interfaces to row i_y + 1.
"""
import numpy as np
import scipy.sparse as sp

from .gll import gll_nodes_weights, diff_matrix

W, E, S, N = 0, 1, 2, 3
OPPOSITE = {W: E, E: W, S: N, N: S}


class SMPMGrid:
    """Geometry, indexing and operators of one SMPM grid."""

    def __init__(self, mx, my, n, Lx=1.0, Ly=1.0, tau_scale=1.0, robin_scale=0.25, robin_literal=False,
                 xs=None, ys=None):
        """Uniform grid of m_x x m_y elements on [0, L_x] x [0, L_y], or, with the
        column edges xs (m_x + 1 increasing values) and row edges ys (m_y + 1),
        the graded grid on [xs[0], xs[-1]] x [ys[0], ys[-1]]."""
        if mx < 1 or my < 1 or n < 2:
            raise ValueError("bad grid")
        self.mx, self.my, self.n = int(mx), int(my), int(n)
        self.tau_scale = float(tau_scale)
        self.robin_scale = float(robin_scale)
        self.robin_literal = bool(robin_literal)
        self.x1d, self.w1d = gll_nodes_weights(self.n)
        self.D = diff_matrix(self.x1d)
        self.graded = xs is not None or ys is not None
        self.xe = self._edges(xs, self.mx, float(Lx))
        self.ye = self._edges(ys, self.my, float(Ly))
        self.Lx = float(Lx) if xs is None else self.xe[-1] - self.xe[0]
        self.Ly = float(Ly) if ys is None else self.ye[-1] - self.ye[0]
        self.hxe, self.hye = np.diff(self.xe), np.diff(self.ye)
        if xs is None:
            self.hxe[:] = self.Lx / self.mx
        if ys is None:
            self.hye[:] = self.Ly / self.my
        # uniform spacing (None on a graded grid: every use goes through h_of)
        self.hx = None if xs is not None else self.Lx / self.mx
        self.hy = None if ys is not None else self.Ly / self.my
        self.nel = self.mx * self.my
        self.nn = self.n * self.n
        self.r = self.nn * self.nel
        self.kp = 4 * self.n * self.nel
        self._build_slots()

    @staticmethod
    def _edges(edges, m, L):
        if edges is None:
            return np.arange(m + 1) * (L / m)
        e = np.asarray(edges, dtype=np.float64)
        if e.shape != (m + 1,) or not np.all(np.diff(e) > 0):
            raise ValueError("element edges must be m + 1 increasing values")
        return e.copy()

    # ---------------------------------------------------------------- indexing
    def element(self, ix, iy):
        return iy * self.mx + ix

    def element_ij(self, e):
        return e % self.mx, e // self.mx

    def neighbour(self, e, F):
        """Element across face F of e, or -1 on the physical boundary."""
        ix, iy = self.element_ij(e)
        jx, jy = {W: (ix - 1, iy), E: (ix + 1, iy), S: (ix, iy - 1), N: (ix, iy + 1)}[F]
        if 0 <= jx < self.mx and 0 <= jy < self.my:
            return self.element(jx, jy)
        return -1

    def face_node(self, F, t):
        """(a, b) of face node t of face F."""
        n = self.n
        return {W: (0, t), E: (n - 1, t), S: (t, 0), N: (t, n - 1)}[F]

    def node(self, e, a, b):
        return e * self.nn + b * self.n + a

    def h_of(self, e):
        """(h_x, h_y) of element e."""
        ix, iy = self.element_ij(e)
        return self.hxe[ix], self.hye[iy]

    def h_perp(self, F, e):
        """Size of element e across face F: h_x for W/E faces, h_y for S/N."""
        hx, hy = self.h_of(e)
        return hx if F in (W, E) else hy

    def tau(self, F, e):
        """Penalty tau_F of face F of element e, Eq. (smpm_poisson) (reading:
        -alpha n(n-1)/h_perp)."""
        return -self.tau_scale * self.n * (self.n - 1) / self.h_perp(F, e)

    def robin_weight(self, F, e):
        """Weight p_F of the identity in the Robin flux R of face F of element e
        (Sec. 1.2) (reading: beta n(n-1)/h_perp; 1 under the literal reading
        R = I + n.grad)."""
        if self.robin_literal:
            return 1.0
        return self.robin_scale * self.n * (self.n - 1) / self.h_perp(F, e)

    def _build_slots(self):
        n = self.n
        self.interfaces = []            # (e, F) with F in {E, N}: the W/S side is the neighbour
        for iy in range(self.my):
            for ix in range(self.mx - 1):
                self.interfaces.append((self.element(ix, iy), E))
            if iy < self.my - 1:
                for ix in range(self.mx):
                    self.interfaces.append((self.element(ix, iy), N))
        self.d = len(self.interfaces)
        iface_of = {}
        for j, (e, F) in enumerate(self.interfaces):
            iface_of[(e, F)] = j
            iface_of[(self.neighbour(e, F), OPPOSITE[F])] = j
        self.iface_of = iface_of
        slots = []                      # real slots (e, F, t) in padded order
        for e in range(self.nel):
            for F in (W, E, S, N):
                if self.neighbour(e, F) >= 0:
                    for t in range(n):
                        slots.append((e, F, t))
        self.slots = slots
        self.k = len(slots)
        self.padded_index = np.array([e * 4 * n + F * n + t for (e, F, t) in slots], dtype=np.int64)
        self.slot_of = {s: i for i, s in enumerate(slots)}

    def to_padded(self, v):
        out = np.zeros(self.kp if v.ndim == 1 else (self.kp,) + v.shape[1:])
        out[self.padded_index] = v
        return out

    def from_padded(self, vp):
        return np.asarray(vp)[self.padded_index]

    # ------------------------------------------------------------- geometry
    def coords(self):
        """Physical x, y of every node (element map of Sec. 1.2 / Sec. 3)."""
        x = np.empty(self.r)
        y = np.empty(self.r)
        for e in range(self.nel):
            ix, iy = self.element_ij(e)
            hx, hy = self.h_of(e)
            for b in range(self.n):
                for a in range(self.n):
                    q = self.node(e, a, b)
                    x[q] = self.xe[ix] + (self.x1d[a] + 1.0) * hx / 2.0
                    y[q] = self.ye[iy] + (self.x1d[b] + 1.0) * hy / 2.0
        return x, y

    def mass(self):
        """GLL quadrature weight W_q = w_a w_b h_x h_y / 4 of every node."""
        m = np.empty(self.r)
        for e in range(self.nel):
            hx, hy = self.h_of(e)
            for b in range(self.n):
                for a in range(self.n):
                    m[self.node(e, a, b)] = self.w1d[a] * self.w1d[b] * hx * hy / 4.0
        return m

    # ---------------------------------------------------- element operators
    def laplacian_block(self, e):
        """n^2 x n^2 Laplacian of element e: (2/h_x)^2 D^2 along a plus (2/h_y)^2 D^2 along b."""
        I = np.eye(self.n)
        D2 = self.D @ self.D
        hx, hy = self.h_of(e)
        return (2.0 / hx) ** 2 * np.kron(I, D2) + (2.0 / hy) ** 2 * np.kron(D2, I)

    def normal_derivative_row(self, F, t, e):
        """Row vector (over element e's n^2 nodes) of n_F . grad u at face node t of F."""
        n = self.n
        row = np.zeros(self.nn)
        hx, hy = self.h_of(e)
        sx, sy = 2.0 / hx, 2.0 / hy
        if F == W:
            row[t * n + np.arange(n)] = -sx * self.D[0]
        elif F == E:
            row[t * n + np.arange(n)] = sx * self.D[n - 1]
        elif F == S:
            row[np.arange(n) * n + t] = -sy * self.D[0]
        else:
            row[np.arange(n) * n + t] = sy * self.D[n - 1]
        return row

    def robin_row(self, F, t, e):
        """R u = p_F u + n_F . grad u at face node t of face F of element e, as a
        row over e's nodes (R_ii of Sec. 1.2)."""
        row = self.normal_derivative_row(F, t, e)
        a, b = self.face_node(F, t)
        row[b * self.n + a] += self.robin_weight(F, e)
        return row

    def neighbour_robin_row(self, F, t, e):
        """(p_F u' + n_F . grad u') at the node of the neighbour e' across face F
        of e that coincides with face node t of F, as a row over e''s nodes.
        p_F is e's (the same R acts on both traces); n_F is e's outward
        normal, i.e. minus e''s own normal on its face opposite(F), and the
        gradient is taken with e''s own map."""
        G = OPPOSITE[F]
        row = -self.normal_derivative_row(G, t, self.neighbour(e, F))
        a, b = self.face_node(G, t)
        row[b * self.n + a] += self.robin_weight(F, e)
        return row

    # ------------------------------------------------------ global operators
    def assemble_L(self):
        """The SMPM operator L (r x r) of Eq. (smpm_poisson):
        L_i u_i = lap u_i + tau_i (R_ii u_i - sum_j R_ij u_j) on interface faces
                  + tau_i n.grad u_i on boundary faces."""
        rows, cols, vals = [], [], []
        nn = self.nn
        loc = np.arange(nn)
        for e in range(self.nel):
            o = e * nn
            lap = self.laplacian_block(e)
            rr, cc = np.nonzero(lap)
            rows.append(o + rr); cols.append(o + cc); vals.append(lap[rr, cc])
            for F in (W, E, S, N):
                e2 = self.neighbour(e, F)
                tau = self.tau(F, e)
                for t in range(self.n):
                    a, b = self.face_node(F, t)
                    q = self.node(e, a, b)
                    if e2 >= 0:
                        own = tau * self.robin_row(F, t, e)
                        nb = -tau * self.neighbour_robin_row(F, t, e)
                        rows.append(np.full(nn, q)); cols.append(o + loc); vals.append(own)
                        rows.append(np.full(nn, q)); cols.append(e2 * nn + loc); vals.append(nb)
                    else:
                        own = tau * self.normal_derivative_row(F, t, e)
                        rows.append(np.full(nn, q)); cols.append(o + loc); vals.append(own)
        Lm = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(self.r, self.r)).tocsr()
        Lm.eliminate_zeros()
        return Lm

    def element_A(self, e):
        """Local block A_e (Sec. 1.3): Laplacian, boundary term and R_ii terms of element e."""
        A = self.laplacian_block(e).copy()
        for F in (W, E, S, N):
            tau = self.tau(F, e)
            interface = self.neighbour(e, F) >= 0
            for t in range(self.n):
                a, b = self.face_node(F, t)
                q = b * self.n + a
                A[q] += tau * (self.robin_row(F, t, e) if interface else self.normal_derivative_row(F, t, e))
        return A

    def assemble_B(self):
        """Flux operator B: Omega -> Gamma (k x r, Sec. 1.3):
        (B u)_(e,F,t) = -tau_F (p_F u' + n_F.grad u')(q'), u' the neighbour across F
        and tau_F, p_F those of e's face F."""
        rows, cols, vals = [], [], []
        loc = np.arange(self.nn)
        for i, (e, F, t) in enumerate(self.slots):
            e2 = self.neighbour(e, F)
            rows.append(np.full(self.nn, i)); cols.append(e2 * self.nn + loc)
            vals.append(-self.tau(F, e) * self.neighbour_robin_row(F, t, e))
        Bm = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(self.k, self.r)).tocsr()
        Bm.eliminate_zeros()
        return Bm

    def assemble_E(self):
        """Inclusion E: Gamma -> Omega (r x k, 0/1, Sec. 1.3): slot (e,F,t) -> its face node."""
        rows = []
        for (e, F, t) in self.slots:
            a, b = self.face_node(F, t)
            rows.append(self.node(e, a, b))
        return sp.csr_matrix((np.ones(self.k), (np.array(rows), np.arange(self.k))),
                             shape=(self.r, self.k))

    def rhs(self, f, g=None):
        """b = f + tau g (Eq. smpm_poisson).  g is given per padded slot; only
        slots on physical-boundary faces are read; a corner node on two
        boundary faces receives both faces' terms."""
        b = np.array(f, dtype=np.float64, copy=True)
        if g is None:
            return b
        g = np.asarray(g, dtype=np.float64)
        for e in range(self.nel):
            for F in (W, E, S, N):
                if self.neighbour(e, F) >= 0:
                    continue
                for t in range(self.n):
                    a, b_ = self.face_node(F, t)
                    b[self.node(e, a, b_)] += self.tau(F, e) * g[e * 4 * self.n + F * self.n + t]
        return b

    def boundary_g(self, gfun):
        """Padded slot array of g = gfun(x, y, nx, ny) on physical-boundary faces."""
        x, y = self.coords()
        g = np.zeros(self.kp)
        normals = {W: (-1.0, 0.0), E: (1.0, 0.0), S: (0.0, -1.0), N: (0.0, 1.0)}
        for e in range(self.nel):
            for F in (W, E, S, N):
                if self.neighbour(e, F) >= 0:
                    continue
                for t in range(self.n):
                    a, b = self.face_node(F, t)
                    q = self.node(e, a, b)
                    g[e * 4 * self.n + F * self.n + t] = gfun(x[q], y[q], *normals[F])
        return g

    def zero_mean(self, u):
        """Remove the GLL-quadrature-weighted mean (the constant left undetermined
        by the Neumann problem, Sec. 1.4)."""
        m = self.mass()
        return u - (m @ u) / m.sum()
