"""The SMPM operator L of Eq. smpm_poisson (Sec. 1.2) computed a second way,
for pinning the oracle: each column of L is the residual of one nodal basis
function, a product of Lagrange polynomials written in PHYSICAL coordinates
and differentiated as polynomials (numpy.polynomial), evaluated at the
physical points of the nodes.  Nothing here uses a differentiation matrix,
the oracle's node tables or its face-node matching: the neighbour's value and
gradient at a face node are the neighbour's polynomial evaluated at that
point.  The GLL nodes are the closed forms for n <= 5 (roots of P'_{n-1}).

The face terms follow Eq. smpm_poisson with R = p_F I + n.grad and the
readings of the penalty and the Robin weight:
    tau_F = -tau_scale n(n-1)/h_perp,
    p_F   = robin_scale n(n-1)/h_perp   (or 1 under the literal R = I + n.grad),
h_perp = h_x on W/E faces, h_y on S/N faces, of the element whose residual row
it is (graded grids: column edges xs, row edges ys).
"""
import numpy as np
from numpy.polynomial import Polynomial

GLL_CLOSED_FORM = {
    2: [-1.0, 1.0],
    3: [-1.0, 0.0, 1.0],
    4: [-1.0, -1.0 / np.sqrt(5.0), 1.0 / np.sqrt(5.0), 1.0],
    5: [-1.0, -np.sqrt(3.0 / 7.0), 0.0, np.sqrt(3.0 / 7.0), 1.0],
}


def _lagrange(nodes, a):
    others = [c for i, c in enumerate(nodes) if i != a]
    return Polynomial.fromroots(others) / np.prod([nodes[a] - c for c in others])


def operator_by_polynomials(mx, my, n, Lx, Ly, tau_scale=1.0, robin_scale=0.25, literal=False,
                            xs=None, ys=None):
    """Dense r x r L, node (a, b) of element e = iy*mx + ix at e*n*n + b*n + a.
    xs / ys: column / row edges of a graded grid (else uniform on [0,Lx]x[0,Ly])."""
    xi = np.array(GLL_CLOSED_FORM[n])
    xe = np.linspace(0.0, Lx, mx + 1) if xs is None else np.asarray(xs, float)
    ye = np.linspace(0.0, Ly, my + 1) if ys is None else np.asarray(ys, float)
    nel, nn = mx * my, n * n
    r = nel * nn

    def sizes(e):
        ix, iy = e % mx, e // mx
        return xe[ix + 1] - xe[ix], ye[iy + 1] - ye[iy]

    # physical node coordinates and the 1-D Lagrange bases of every element
    def elem_nodes(e):
        ix, iy = e % mx, e // mx
        hx, hy = sizes(e)
        return xe[ix] + (xi + 1) * hx / 2, ye[iy] + (xi + 1) * hy / 2

    bases = []
    for e in range(nel):
        xs, ys = elem_nodes(e)
        lx = [_lagrange(xs, a) for a in range(n)]
        ly = [_lagrange(ys, b) for b in range(n)]
        bases.append((lx, ly))

    def neighbour(e, F):
        ix, iy = e % mx, e // mx
        jx, jy = {0: (ix - 1, iy), 1: (ix + 1, iy), 2: (ix, iy - 1), 3: (ix, iy + 1)}[F]
        return jy * mx + jx if (0 <= jx < mx and 0 <= jy < my) else -1

    normal = {0: (-1.0, 0.0), 1: (1.0, 0.0), 2: (0.0, -1.0), 3: (0.0, 1.0)}

    def value_grad_lap(e, a, b, x, y):
        """phi_(e,a,b), its gradient and Laplacian at the point (x, y)."""
        lx, ly = bases[e]
        px, py = lx[a], ly[b]
        v = px(x) * py(y)
        gx = px.deriv()(x) * py(y)
        gy = px(x) * py.deriv()(y)
        lap = px.deriv(2)(x) * py(y) + px(x) * py.deriv(2)(y)
        return v, gx, gy, lap

    L = np.zeros((r, r))
    for e in range(nel):
        xs, ys = elem_nodes(e)
        for b in range(n):
            for a in range(n):
                row = e * nn + b * n + a
                x, y = xs[a], ys[b]
                faces = [F for F, on in ((0, a == 0), (1, a == n - 1), (2, b == 0), (3, b == n - 1)) if on]
                # columns: basis functions of e and of its neighbours
                for ec in [e] + [neighbour(e, F) for F in range(4) if neighbour(e, F) >= 0]:
                    for bc in range(n):
                        for ac in range(n):
                            col = ec * nn + bc * n + ac
                            v, gx, gy, lap = value_grad_lap(ec, ac, bc, x, y)
                            own = ec == e
                            val = lap if own else 0.0
                            for F in faces:
                                hp = sizes(e)[0] if F in (0, 1) else sizes(e)[1]
                                tau = -tau_scale * n * (n - 1) / hp
                                p = 1.0 if literal else robin_scale * n * (n - 1) / hp
                                nx, ny = normal[F]
                                dn = nx * gx + ny * gy
                                e2 = neighbour(e, F)
                                if e2 < 0:
                                    if own:
                                        val += tau * dn
                                elif own:
                                    val += tau * (p * v + dn)
                                elif ec == e2:
                                    val -= tau * (p * v + dn)
                            L[row, col] += val
    return L


def read_golden_n2(path):
    """Entries of the hand-derived n = 2 operators: {grid: [(row, col, cXX, cYY, cXP, cYP)]}."""
    out = {}
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            g, *nums = line.split()
            i, j, cxx, cyy, cxp, cyp = (int(t) for t in nums)
            out.setdefault(g, []).append((i, j, cxx, cyy, cxp, cyp))
    return out


def golden_matrix(entries, hx, hy, px, py):
    X, Y = 1.0 / hx, 1.0 / hy
    Lg = np.zeros((8, 8))
    for i, j, cxx, cyy, cxp, cyp in entries:
        Lg[i, j] = cxx * X * X + cyy * Y * Y + cxp * X * px + cyp * Y * py
    return Lg
