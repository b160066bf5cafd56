"""SMPM discretisation of the 2-D Poisson-Neumann problem (Sec. 1.2 - 1.3).

Conventions fixed here (the paper leaves them open; each is a reading of the
passage cited):

* Elements: an m_y x m_x Cartesian grid on [0, L_x] x [0, L_y] (Sec. 1.2, Sec. 3),
  element e = i_y * m_x + i_x covering [i_x h_x, (i_x+1) h_x] x [i_y h_y, (i_y+1) h_y].
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

    def __init__(self, mx, my, n, Lx=1.0, Ly=1.0, tau_scale=1.0, robin_scale=0.25, robin_literal=False):
        if mx < 1 or my < 1 or n < 2:
            raise ValueError("bad grid")
        self.mx, self.my, self.n = int(mx), int(my), int(n)
        self.Lx, self.Ly = float(Lx), float(Ly)
        self.tau_scale = float(tau_scale)
        self.robin_scale = float(robin_scale)
        self.robin_literal = bool(robin_literal)
        self.x1d, self.w1d = gll_nodes_weights(self.n)
        self.D = diff_matrix(self.x1d)
        self.hx, self.hy = self.Lx / self.mx, self.Ly / self.my
        self.nel = self.mx * self.my
        self.nn = self.n * self.n
        self.r = self.nn * self.nel
        self.kp = 4 * self.n * self.nel
        self._build_slots()

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

    def tau(self, F):
        """Penalty tau_F of Eq. (smpm_poisson) (reading: -alpha n(n-1)/h_perp)."""
        h = self.hx if F in (W, E) else self.hy
        return -self.tau_scale * self.n * (self.n - 1) / h

    def robin_weight(self, F):
        """Weight p_F of the identity in the Robin flux R of Sec. 1.2 (reading:
        beta n(n-1)/h_perp; 1 under the literal reading R = I + n.grad)."""
        if self.robin_literal:
            return 1.0
        h = self.hx if F in (W, E) else self.hy
        return self.robin_scale * self.n * (self.n - 1) / h

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
            for b in range(self.n):
                for a in range(self.n):
                    q = self.node(e, a, b)
                    x[q] = ix * self.hx + (self.x1d[a] + 1.0) * self.hx / 2.0
                    y[q] = iy * self.hy + (self.x1d[b] + 1.0) * self.hy / 2.0
        return x, y

    def mass(self):
        """GLL quadrature weight W_q = w_a w_b h_x h_y / 4 of every node."""
        m = np.empty(self.r)
        for e in range(self.nel):
            for b in range(self.n):
                for a in range(self.n):
                    m[self.node(e, a, b)] = self.w1d[a] * self.w1d[b] * self.hx * self.hy / 4.0
        return m

    # ---------------------------------------------------- element operators
    def laplacian_block(self):
        """n^2 x n^2 element Laplacian: (2/h_x)^2 D^2 along a plus (2/h_y)^2 D^2 along b."""
        I = np.eye(self.n)
        D2 = self.D @ self.D
        return (2.0 / self.hx) ** 2 * np.kron(I, D2) + (2.0 / self.hy) ** 2 * np.kron(D2, I)

    def normal_derivative_row(self, F, t):
        """Row vector (over one element's n^2 nodes) of n_F . grad u at face node t of F."""
        n = self.n
        row = np.zeros(self.nn)
        sx, sy = 2.0 / self.hx, 2.0 / self.hy
        if F == W:
            row[t * n + np.arange(n)] = -sx * self.D[0]
        elif F == E:
            row[t * n + np.arange(n)] = sx * self.D[n - 1]
        elif F == S:
            row[np.arange(n) * n + t] = -sy * self.D[0]
        else:
            row[np.arange(n) * n + t] = sy * self.D[n - 1]
        return row

    def robin_row(self, F, t):
        """R u = p_F u + n_F . grad u at face node t of face F, as a row over
        one element (R_ii of Sec. 1.2)."""
        row = self.normal_derivative_row(F, t)
        a, b = self.face_node(F, t)
        row[b * self.n + a] += self.robin_weight(F)
        return row

    def neighbour_robin_row(self, F, t):
        """(p_F u' + n_F . grad u') at the node of the neighbour across face F that
        coincides with face node t of F, as a row over the neighbour's nodes.
        n_F is the receiving element's outward normal, i.e. minus the
        neighbour's own normal on its face opposite(F)."""
        G = OPPOSITE[F]
        row = -self.normal_derivative_row(G, t)
        a, b = self.face_node(G, t)
        row[b * self.n + a] += self.robin_weight(F)
        return row

    # ------------------------------------------------------ global operators
    def assemble_L(self):
        """The SMPM operator L (r x r) of Eq. (smpm_poisson):
        L_i u_i = lap u_i + tau_i (R_ii u_i - sum_j R_ij u_j) on interface faces
                  + tau_i n.grad u_i on boundary faces."""
        rows, cols, vals = [], [], []
        lap = self.laplacian_block()
        nn = self.nn
        loc = np.arange(nn)
        for e in range(self.nel):
            o = e * nn
            rr, cc = np.nonzero(lap)
            rows.append(o + rr); cols.append(o + cc); vals.append(lap[rr, cc])
            for F in (W, E, S, N):
                e2 = self.neighbour(e, F)
                tau = self.tau(F)
                for t in range(self.n):
                    a, b = self.face_node(F, t)
                    q = self.node(e, a, b)
                    if e2 >= 0:
                        own = tau * self.robin_row(F, t)
                        nb = -tau * self.neighbour_robin_row(F, t)
                        rows.append(np.full(nn, q)); cols.append(o + loc); vals.append(own)
                        rows.append(np.full(nn, q)); cols.append(e2 * nn + loc); vals.append(nb)
                    else:
                        own = tau * self.normal_derivative_row(F, t)
                        rows.append(np.full(nn, q)); cols.append(o + loc); vals.append(own)
        Lm = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(self.r, self.r)).tocsr()
        Lm.eliminate_zeros()
        return Lm

    def element_A(self, e):
        """Local block A_e (Sec. 1.3): Laplacian, boundary term and R_ii terms of element e."""
        A = self.laplacian_block().copy()
        for F in (W, E, S, N):
            tau = self.tau(F)
            interface = self.neighbour(e, F) >= 0
            for t in range(self.n):
                a, b = self.face_node(F, t)
                q = b * self.n + a
                A[q] += tau * (self.robin_row(F, t) if interface else self.normal_derivative_row(F, t))
        return A

    def assemble_B(self):
        """Flux operator B: Omega -> Gamma (k x r, Sec. 1.3):
        (B u)_(e,F,t) = -tau_F (p_F u' + n_F.grad u')(q'), u' the neighbour across F."""
        rows, cols, vals = [], [], []
        loc = np.arange(self.nn)
        for i, (e, F, t) in enumerate(self.slots):
            e2 = self.neighbour(e, F)
            rows.append(np.full(self.nn, i)); cols.append(e2 * self.nn + loc)
            vals.append(-self.tau(F) * self.neighbour_robin_row(F, t))
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
                    b[self.node(e, a, b_)] += self.tau(F) * g[e * 4 * self.n + F * self.n + t]
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
