"""Algorithm 3 on the Schur system of one grid split over gloo ranks by the
library's element-tile partition (smpm_partition_tile / smpm_partition_halo),
for testing the partition on the CPU.

Each rank keeps full-length padded slot vectors but computes only the slots
of its own elements; everything it needs from other tiles comes through the
exchanges the partition names:

* S v (push form, Eq. schur_complement_system): the products T_e v_e destined
  for a peer's slots (`facing`) are sent; the peer adds them to its `own`;
* M^-1 v (Fig. 2 blocks in the reduced form G = (I - X Y)^-1): a black block
  on a cut reads the peer's values at `facing` and sends its results back;
* P, Q (Eqs. projection1/2): the weighted interface sums Z^T v are partial on
  each rank and all-reduced; the coarse solve H = C^+ is replicated;
* the Gram-Schmidt dot products are all-reduced.

The factors come from the library's host factor step (the same numbers the
device path uploads); the arithmetic here is plain numpy.
"""
import numpy as np
import torch
import torch.distributed as dist

OPP = (1, 0, 3, 2)


class ShardedSchur:
    def __init__(self, lg, px, py, rank):
        self.px, self.py, self.rank = px, py, rank
        self.mx, self.my, self.n = lg.mx, lg.my, lg.n
        n, M = lg.n, 4 * lg.n
        self.M, self.kp, self.d = M, lg.kp, lg.d
        self.tile = lg.partition_tile(px, py, rank)
        t = self.tile
        self.owned = [iy * lg.mx + ix for iy in range(t["iy0"], t["iy1"]) for ix in range(t["ix0"], t["ix1"])]
        self.owned_set = set(self.owned)
        self.own_slots = np.concatenate([np.arange(e * M, (e + 1) * M) for e in self.owned])
        self.sides = []
        for side in range(4):
            if t["peers"][side] >= 0:
                own, facing = lg.partition_halo(px, py, rank, side)
                self.sides.append((side, t["peers"][side], own, facing))
        nel = lg.mx * lg.my
        self.T = lg.host_factor("T").reshape(nel, M, M)
        self.G = lg.host_factor("G").reshape(-1, M, M)
        self.X = lg.host_factor("X").reshape(-1, 4, n, n)
        self.black = [int(b) for b in lg.host_factor("black")]
        self.block_of = {e: ib for ib, e in enumerate(self.black)}
        self.Rs = lg.host_factor("Rs").reshape(nel, M, 4)
        self.H = lg.host_factor("H").reshape(lg.d, lg.d)
        self.zw = lg.host_factor("zw").reshape(nel, 4)
        self.exchanged = 0   # values sent by this rank

    # ------------------------------------------------------------ geometry
    def nbr(self, e, F):
        ix, iy = e % self.mx, e // self.mx
        if F == 0:
            return e - 1 if ix > 0 else -1
        if F == 1:
            return e + 1 if ix < self.mx - 1 else -1
        if F == 2:
            return e - self.mx if iy > 0 else -1
        return e + self.mx if iy < self.my - 1 else -1

    def iface(self, e, F):
        ix, iy, row = e % self.mx, e // self.mx, 2 * self.mx - 1
        if F == 0:
            return iy * row + ix - 1 if ix > 0 else -1
        if F == 1:
            return iy * row + ix if ix < self.mx - 1 else -1
        if F == 2:
            return (iy - 1) * row + self.mx - 1 + ix if iy > 0 else -1
        return iy * row + self.mx - 1 + ix if iy < self.my - 1 else -1

    def is_black(self, e):
        return ((e % self.mx) + (e // self.mx)) % 2 == 0

    # ---------------------------------------------------------- exchanges
    def swap(self, values_by_side):
        """Send values_by_side[side] to that side's peer; return what each peer
        sent back, by side (point-to-point, deadlock-free ordering by rank)."""
        out = {}
        for side, peer, own, facing in self.sides:
            buf = torch.as_tensor(np.ascontiguousarray(values_by_side[side]))
            rcv = torch.empty_like(buf)
            if self.rank < peer:
                dist.send(buf, peer)
                dist.recv(rcv, peer)
            else:
                dist.recv(rcv, peer)
                dist.send(buf, peer)
            self.exchanged += buf.numel()
            out[side] = rcv.numpy()
        return out

    def allreduce(self, arr):
        buf = torch.as_tensor(np.ascontiguousarray(arr, dtype=np.float64))
        dist.all_reduce(buf)
        return buf.numpy()

    def dot(self, a, b):
        return float(self.allreduce(np.array([a[self.own_slots] @ b[self.own_slots]]))[0])

    # ---------------------------------------------------------- operators
    def apply_S(self, v):
        """y = S v on the owned slots: y = v + scatter(T_e v_e), push form."""
        n, M = self.n, self.M
        push = np.zeros(self.kp)
        for e in self.owned:
            z = self.T[e] @ v[e * M:(e + 1) * M]
            for F in range(4):
                e2 = self.nbr(e, F)
                if e2 >= 0:
                    push[e2 * M + OPP[F] * n: e2 * M + OPP[F] * n + n] += z[F * n:(F + 1) * n]
        y = np.zeros(self.kp)
        y[self.own_slots] = v[self.own_slots] + push[self.own_slots]
        got = self.swap({side: push[facing] for side, _, _, facing in self.sides})
        for side, _, own, _ in self.sides:
            y[own] += got[side]
        return y

    def apply_Minv(self, v):
        """t = M^-1 v: a = G (p - X q), b = q - T_e a per black block (Fig. 2),
        q the neighbours' slots facing the black element."""
        n, M = self.n, self.M
        vf = v.copy()
        got = self.swap({side: v[own] for side, _, own, _ in self.sides})
        for side, _, _, facing in self.sides:
            vf[facing] = got[side]              # the peer's slots facing this tile
        t = np.zeros(self.kp)
        for e in self.owned:
            if not self.is_black(e):
                continue
            ib = self.block_of[e]
            p = vf[e * M:(e + 1) * M]
            q = np.zeros(M)
            for F in range(4):
                e2 = self.nbr(e, F)
                if e2 >= 0:
                    q[F * n:(F + 1) * n] = vf[e2 * M + OPP[F] * n: e2 * M + OPP[F] * n + n]
            Xq = np.concatenate([self.X[ib, F] @ q[F * n:(F + 1) * n] for F in range(4)])
            a = self.G[ib] @ (p - Xq)
            b = q - self.T[e] @ a
            t[e * M:(e + 1) * M] = a
            for F in range(4):
                e2 = self.nbr(e, F)
                if e2 >= 0:
                    t[e2 * M + OPP[F] * n: e2 * M + OPP[F] * n + n] = b[F * n:(F + 1) * n]
        got = self.swap({side: t[facing] for side, _, _, facing in self.sides})
        for side, _, own, _ in self.sides:
            for k, s in enumerate(own):
                if not self.is_black(int(s) // M):   # the peer's black block wrote it
                    t[s] = got[side][k]
        return t

    def zt(self, v):
        """Z^T v (weighted interface sums), all-reduced over the ranks."""
        n, M = self.n, self.M
        c = np.zeros(self.d)
        for e in self.owned:
            for F in range(4):
                j = self.iface(e, F)
                if j >= 0:
                    c[j] += self.zw[e, F] * v[e * M + F * n: e * M + F * n + n].sum()
        return self.allreduce(c)

    def szc(self, chat):
        """(S Z chat) on the owned slots, pull form: the slot's own weight times
        chat_j plus the weighted row sums of the neighbour's T facing it."""
        n, M = self.n, self.M
        out = np.zeros(self.kp)
        for e in self.owned:
            for F in range(4):
                e2 = self.nbr(e, F)
                if e2 < 0:
                    continue
                j = self.iface(e, F)
                for s in range(n):
                    acc = self.zw[e, F] * chat[j]
                    row = self.Rs[e2, OPP[F] * n + s]
                    for G in range(4):
                        jj = self.iface(e2, G)
                        if jj >= 0:
                            acc += row[G] * chat[jj]
                    out[e * M + F * n + s] = acc
        return out

    def apply_P(self, y):
        return y - self.szc(self.H @ self.zt(y))

    def apply_Q(self, x):
        n, M = self.n, self.M
        chat = self.H @ self.zt(self.apply_S(x))
        return x - self.zc(chat)

    def zc(self, chat):
        """Z chat on the owned slots."""
        n, M = self.n, self.M
        out = np.zeros(self.kp)
        for e in self.owned:
            for F in range(4):
                j = self.iface(e, F)
                if j >= 0:
                    out[e * M + F * n: e * M + F * n + n] = self.zw[e, F] * chat[j]
        return out

    # ---------------------------------------------------------- the solve
    def gmres(self, op, b, tol, restart=50, maxit=1000):
        """Right-preconditioned GMRES(m) with modified Gram-Schmidt; every inner
        product is all-reduced."""
        x = np.zeros(self.kp)
        beta0 = np.sqrt(self.dot(b, b))
        its = 0
        r = b.copy()
        while its < maxit:
            beta = np.sqrt(self.dot(r, r))
            if beta <= tol * beta0:
                break
            V = [r / beta]
            Hm = np.zeros((restart + 1, restart))
            g = np.zeros(restart + 1)
            g[0] = beta
            cs, sn = np.zeros(restart), np.zeros(restart)
            k = 0
            for k in range(restart):
                w = op(V[k])
                for i in range(k + 1):
                    Hm[i, k] = self.dot(w, V[i])
                    w = w - Hm[i, k] * V[i]
                hnext = np.sqrt(self.dot(w, w))
                Hm[k + 1, k] = hnext
                for i in range(k):
                    a, b2 = Hm[i, k], Hm[i + 1, k]
                    Hm[i, k], Hm[i + 1, k] = cs[i] * a + sn[i] * b2, -sn[i] * a + cs[i] * b2
                den = np.hypot(Hm[k, k], Hm[k + 1, k])
                cs[k], sn[k] = Hm[k, k] / den, Hm[k + 1, k] / den
                Hm[k, k], Hm[k + 1, k] = den, 0.0
                g[k + 1] = -sn[k] * g[k]
                g[k] = cs[k] * g[k]
                its += 1
                if abs(g[k + 1]) <= tol * beta0 or its >= maxit:
                    break
                V.append(w / hnext)
            m = k + 1
            yk = np.linalg.solve(np.triu(Hm[:m, :m]), g[:m])
            for i in range(m):
                x = x + yk[i] * V[i]
            r = b - op(x)
        return x, its

    def algorithm3(self, bS, tol=1e-11):
        """x_S = Q M^-1 y + Z C^+ Z^T b_S with y from GMRES(P S M^-1, P b_S)
        (Eq. deflated_schur)."""
        op = lambda v: self.apply_P(self.apply_S(self.apply_Minv(v)))
        y, its = self.gmres(op, self.apply_P(bS), tol)
        x = self.apply_Q(self.apply_Minv(y)) + self.zc(self.H @ self.zt(bS))
        return x, its

    def gather(self, v):
        """The full vector from every rank's owned slots (all-reduce of disjoint parts)."""
        part = np.zeros(self.kp)
        part[self.own_slots] = v[self.own_slots]
        return self.allreduce(part)
