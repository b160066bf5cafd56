"""ctypes binding of libsmpm.so (argument marshalling only).

Every computation runs inside the C ABI declared in ``include/smpm.h``; this
module converts Python/NumPy/PyTorch arguments into plain pointers and sizes.
Loading fails loudly when the library has not been built: there is no CPU
fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmpm.so")

FLAG_NO_SMEM_RESIDENCY, FLAG_STREAM_MATRICES, FLAG_ADJOINT, FLAG_WARP_ELEMS, FLAG_ROBIN_LITERAL = 1, 2, 4, 8, 16
FLAG_NO_LOCKSTEP, FLAG_OPERATOR_ONLY = 32, 64

SMPM_OK, SMPM_EINVAL, SMPM_ENOINTERFACE, SMPM_ENOMEM, SMPM_ECUDA, SMPM_ENOTCONV, SMPM_EBREAKDOWN, SMPM_ENAN, \
    SMPM_ESTATE, SMPM_ETIMEOUT = range(10)
STATUS_NAMES = ["OK", "EINVAL", "ENOINTERFACE", "ENOMEM", "ECUDA", "ENOTCONV", "EBREAKDOWN", "ENAN", "ESTATE",
                "ETIMEOUT"]

# every symbol include/smpm.h declares
EXPORTS = [
    "smpm_default_opts", "smpm_setup", "smpm_setup_graded", "smpm_partition_tile", "smpm_partition_halo",
    "smpm_set_apply_kernel", "smpm_autotune_apply",
    "smpm_sizes", "smpm_node_coords", "smpm_node_mass", "schur_factor",
    "schur_solve", "schur_solve_host", "smpm_apply_schur", "smpm_apply_precond", "smpm_apply_schur_precond",
    "smpm_apply_deflation", "smpm_apply_deflation_q", "smpm_schur_rhs", "smpm_recover", "smpm_null_vectors",
    "smpm_coarse_matrix", "smpm_factor_host_only", "smpm_host_factor", "smpm_destroy", "smpm_last_error",
    "smpm_apply_deflation_noalloc", "smpm_apply_schur32", "schur_solve_adjoint",
    "smpm_factor_many", "smpm_batch_create", "smpm_batch_info", "smpm_batch_solve", "smpm_batch_autotune", "smpm_batch_destroy",
    "smpm_batch_task_times", "smpm_batch_apply_schur", "smpm_batch_apply_schur32",
    "smpm_batch_set_apply_kernel", "smpm_set_barrier_spin_limit", "smpm_apply_schur_class",
    "smpm_apply_schur_class32",
]


class SmpmOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("precision", ctypes.c_int), ("precond", ctypes.c_int), ("tau_scale", ctypes.c_double),
                ("robin_scale", ctypes.c_double), ("flags", ctypes.c_int)]


class SmpmReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("refinements", ctypes.c_int),
                ("converged", ctypes.c_int), ("gmres_relres", ctypes.c_double), ("schur_relres", ctypes.c_double),
                ("launches", ctypes.c_int), ("gmres_ms", ctypes.c_double),
                ("pre_ms", ctypes.c_double), ("post_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


APPLY_AUTO, APPLY_WARP, APPLY_WARP2, APPLY_WARP4, APPLY_STREAM, APPLY_CLASS = range(6)


class SmpmTile(ctypes.Structure):
    _fields_ = [("px", ctypes.c_int), ("py", ctypes.c_int), ("rank", ctypes.c_int),
                ("ix0", ctypes.c_int), ("ix1", ctypes.c_int), ("iy0", ctypes.c_int), ("iy1", ctypes.c_int),
                ("nel_owned", ctypes.c_longlong), ("npeers", ctypes.c_int), ("peers", ctypes.c_int * 4),
                ("halo", ctypes.c_longlong * 4)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["peers"], d["halo"] = list(self.peers), list(self.halo)
        return d


class SmpmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


_lib = None


def lib():
    """The loaded libsmpm.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsmpm.so is not built; run __graft_entry__.build() "
                              "(python -m paper_1601_03432_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        L.smpm_default_opts.argtypes = [ctypes.POINTER(SmpmOpts)]
        L.smpm_default_opts.restype = None
        L.smpm_setup.argtypes = [I, I, I, D, D, ctypes.POINTER(P)]
        L.smpm_setup_graded.argtypes = [I, I, I, P, P, ctypes.POINTER(P)]
        L.smpm_partition_tile.argtypes = [P, I, I, I, ctypes.POINTER(SmpmTile)]
        L.smpm_partition_halo.argtypes = [P, I, I, I, I, P, P]
        L.smpm_set_apply_kernel.argtypes = [P, I]
        L.smpm_autotune_apply.argtypes = [P, I, I, I, P, P, P]
        L.smpm_sizes.argtypes = [P] + [ctypes.POINTER(LL)] * 5
        L.smpm_node_coords.argtypes = [P, P, P]
        L.smpm_node_mass.argtypes = [P, P]
        L.schur_factor.argtypes = [P, ctypes.POINTER(SmpmOpts), P]
        L.schur_solve.argtypes = [P, P, P, D, I, P, ctypes.POINTER(SmpmReport), P]
        L.schur_solve_host.argtypes = [P, P, P, D, I, P, ctypes.POINTER(SmpmReport), P]
        L.schur_solve_adjoint.argtypes = [P, P, D, I, P, P, ctypes.POINTER(SmpmReport), P]
        for name in ["smpm_apply_schur", "smpm_apply_precond", "smpm_apply_schur_precond", "smpm_apply_deflation",
                     "smpm_apply_deflation_q", "smpm_schur_rhs", "smpm_apply_deflation_noalloc",
                     "smpm_apply_schur32", "smpm_apply_schur_class", "smpm_apply_schur_class32"]:
            getattr(L, name).argtypes = [P, P, P, P]
        L.smpm_recover.argtypes = [P, P, P, P, P]
        L.smpm_null_vectors.argtypes = [P, P, P, P, P]
        L.smpm_coarse_matrix.argtypes = [P, P]
        L.smpm_factor_host_only.argtypes = [P, ctypes.POINTER(SmpmOpts)]
        L.smpm_host_factor.argtypes = [P, ctypes.c_char_p, P, LL, ctypes.POINTER(LL)]
        L.smpm_destroy.argtypes = [P]
        L.smpm_destroy.restype = None
        L.smpm_factor_many.argtypes = [P, I, ctypes.POINTER(SmpmOpts), P]
        L.smpm_batch_create.argtypes = [P, I, P, I, I, I, ctypes.POINTER(P)]
        L.smpm_batch_info.argtypes = [P, ctypes.POINTER(LL), ctypes.POINTER(LL), ctypes.POINTER(LL),
                                      ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]
        L.smpm_batch_solve.argtypes = [P, P, P, P, ctypes.POINTER(SmpmReport), P]
        L.smpm_batch_autotune.argtypes = [P, P, P, P, P, P, I, P, ctypes.POINTER(I)]
        L.smpm_batch_task_times.argtypes = [P, P, P, P]
        L.smpm_batch_apply_schur.argtypes = [P, P, P, P]
        L.smpm_batch_apply_schur32.argtypes = [P, P, P, P]
        L.smpm_batch_set_apply_kernel.argtypes = [P, I]
        L.smpm_set_barrier_spin_limit.argtypes = [LL]
        L.smpm_batch_destroy.argtypes = [P]
        L.smpm_batch_destroy.restype = None
        L.smpm_last_error.argtypes = []
        L.smpm_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("smpm_default_opts", "smpm_destroy", "smpm_last_error", "smpm_batch_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def check(status, allow=()):
    if status != SMPM_OK and status not in allow:
        raise SmpmError(status, lib().smpm_last_error().decode())
    return status


def default_opts(**kw):
    o = SmpmOpts()
    lib().smpm_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _dev(x, n, name, dtype="float64", optional=False):
    """Pointer of a contiguous CUDA tensor of `dtype` holding at least n
    entries.  The C ABI takes lengths from the handle, so a short, host or
    wrongly typed buffer is refused here rather than read out of bounds."""
    if x is None:
        if optional:
            return None
        raise TypeError("%s: a CUDA tensor is required" % name)
    if isinstance(x, np.ndarray) or not getattr(x, "is_cuda", False):
        raise TypeError("%s: expected a CUDA tensor" % name)
    if str(x.dtype) != "torch." + dtype or not x.is_contiguous():
        raise TypeError("%s: expected a contiguous %s tensor, got %s" % (name, dtype, x.dtype))
    if x.numel() < n:
        raise ValueError("%s: %d entries, %d needed" % (name, x.numel(), n))
    return x.data_ptr()


def _host(x, n, name, optional=False):
    """Pointer of a contiguous float64 NumPy array of at least n entries."""
    if x is None:
        if optional:
            return None
        raise TypeError("%s: a NumPy array is required" % name)
    if not isinstance(x, np.ndarray) or x.dtype != np.float64 or not x.flags.c_contiguous:
        raise TypeError("%s: expected a contiguous float64 NumPy array" % name)
    if x.size < n:
        raise ValueError("%s: %d entries, %d needed" % (name, x.size, n))
    return x.ctypes.data


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


class Grid:
    """One SMPM grid and its factors, owned through an smpm_handle."""

    def __init__(self, mx, my, n, Lx=1.0, Ly=1.0, xs=None, ys=None):
        """Uniform grid on [0,Lx]x[0,Ly], or with column edges xs (mx+1) and/or
        row edges ys (my+1) the graded grid (smpm_setup_graded)."""
        h = ctypes.c_void_p()
        if xs is None and ys is None:
            check(lib().smpm_setup(mx, my, n, float(Lx), float(Ly), ctypes.byref(h)))
        else:
            ex = np.ascontiguousarray(np.arange(mx + 1) * (Lx / mx) if xs is None else xs, dtype=np.float64)
            ey = np.ascontiguousarray(np.arange(my + 1) * (Ly / my) if ys is None else ys, dtype=np.float64)
            if ex.shape != (mx + 1,) or ey.shape != (my + 1,):
                raise ValueError("xs needs mx + 1 and ys my + 1 edges")
            check(lib().smpm_setup_graded(mx, my, n, ex.ctypes.data, ey.ctypes.data, ctypes.byref(h)))
            Lx, Ly = float(ex[-1] - ex[0]), float(ey[-1] - ey[0])
        self.h = h
        self.mx, self.my, self.n, self.Lx, self.Ly = mx, my, n, Lx, Ly
        vals = [ctypes.c_longlong() for _ in range(5)]
        check(lib().smpm_sizes(h, *[ctypes.byref(v) for v in vals]))
        self.r, self.kp, self.d, self.k, self.nblack = [v.value for v in vals]
        self.factored = False

    def close(self):
        if getattr(self, "h", None):
            lib().smpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def node_coords(self):
        x = np.empty(self.r)
        y = np.empty(self.r)
        check(lib().smpm_node_coords(self.h, x.ctypes.data, y.ctypes.data))
        return x, y

    def node_mass(self):
        w = np.empty(self.r)
        check(lib().smpm_node_mass(self.h, w.ctypes.data))
        return w

    def factor(self, stream=None, **opts):
        o = default_opts(**opts)
        check(lib().schur_factor(self.h, ctypes.byref(o), _stream(stream)))
        self.opts = o
        self.factored = True

    def factor_host_only(self, **opts):
        o = default_opts(**opts)
        check(lib().smpm_factor_host_only(self.h, ctypes.byref(o)))

    def set_apply_kernel(self, kind):
        """smpm_set_apply_kernel: one of APPLY_AUTO .. APPLY_CLASS."""
        check(lib().smpm_set_apply_kernel(self.h, int(kind)))

    def autotune_apply(self, precision=0, reps=5, flush=True, stream=None):
        """smpm_autotune_apply: times every available apply kernel, keeps the
        fastest; returns (chosen kind, {kind: median ms})."""
        ms = np.empty(5)
        ch = ctypes.c_int()
        check(lib().smpm_autotune_apply(self.h, int(precision), int(reps), 1 if flush else 0, ms.ctypes.data,
                                        ctypes.byref(ch), _stream(stream)))
        return ch.value, {k + 1: float(ms[k]) for k in range(5) if ms[k] >= 0}

    def partition_tile(self, px, py, rank):
        """smpm_partition_tile: the element tile and the cut sides of rank."""
        t = SmpmTile()
        check(lib().smpm_partition_tile(self.h, px, py, rank, ctypes.byref(t)))
        return t.as_dict()

    def partition_halo(self, px, py, rank, side):
        """smpm_partition_halo: (own, facing) padded slot lists across side."""
        m = self.partition_tile(px, py, rank)["halo"][side]
        own = np.empty(m, dtype=np.int64)
        facing = np.empty(m, dtype=np.int64)
        check(lib().smpm_partition_halo(self.h, px, py, rank, side, own.ctypes.data, facing.ctypes.data))
        return own, facing

    def host_factor(self, name):
        n = ctypes.c_longlong()
        check(lib().smpm_host_factor(self.h, name.encode(), None, 0, ctypes.byref(n)))
        out = np.empty(n.value)
        check(lib().smpm_host_factor(self.h, name.encode(), out.ctypes.data, n.value, None))
        return out

    def coarse_matrix(self):
        C = np.empty((self.d, self.d))
        check(lib().smpm_coarse_matrix(self.h, C.ctypes.data))
        return C

    def solve(self, f, u, g=None, tol=0.0, nrhs=1, stream=None, allow_notconv=False, allow=()):
        """schur_solve on device tensors (float64, contiguous); returns the
        reports.  Statuses in `allow` (and ENOTCONV with allow_notconv) are
        returned in each report's "status" instead of raised."""
        reps = (SmpmReport * nrhs)()
        st = lib().schur_solve(self.h, _dev(f, self.r * nrhs, "f"), _dev(g, self.kp * nrhs, "g", optional=True),
                               float(tol), nrhs, _dev(u, self.r * nrhs, "u"), reps, _stream(stream))
        check(st, allow=tuple(allow) + ((SMPM_ENOTCONV,) if allow_notconv else ()))
        return [dict(r.as_dict(), status=st) for r in reps]

    def solve_adjoint(self, gbar_u, gbar_f, gbar_g=None, tol=0.0, nrhs=1, stream=None, allow_notconv=False):
        """schur_solve_adjoint on device tensors: dl/df (and dl/dg) from dl/du;
        needs factor(flags=FLAG_ADJOINT)."""
        reps = (SmpmReport * nrhs)()
        st = lib().schur_solve_adjoint(self.h, _dev(gbar_u, self.r * nrhs, "gbar_u"), float(tol), nrhs,
                                       _dev(gbar_f, self.r * nrhs, "gbar_f"),
                                       _dev(gbar_g, self.kp * nrhs, "gbar_g", optional=True), reps, _stream(stream))
        check(st, allow=(SMPM_ENOTCONV,) if allow_notconv else ())
        return [r.as_dict() for r in reps]

    def solve_host(self, f, u, g=None, tol=0.0, nrhs=1, stream=None, allow_notconv=False):
        """schur_solve_host on host NumPy arrays."""
        reps = (SmpmReport * nrhs)()
        st = lib().schur_solve_host(self.h, _host(f, self.r * nrhs, "f"), _host(g, self.kp * nrhs, "g", optional=True),
                                    float(tol), nrhs, _host(u, self.r * nrhs, "u"), reps, _stream(stream))
        check(st, allow=(SMPM_ENOTCONV,) if allow_notconv else ())
        return [r.as_dict() for r in reps]

    def _op(self, name, v, out, stream=None, n_in=None, n_out=None, dtype="float64"):
        n_in = self.kp if n_in is None else n_in
        n_out = self.kp if n_out is None else n_out
        check(getattr(lib(), name)(self.h, _dev(v, n_in, "v", dtype), _dev(out, n_out, "out", dtype),
                                   _stream(stream)))
        return out

    def apply_schur(self, v, out, stream=None):
        return self._op("smpm_apply_schur", v, out, stream)

    def apply_schur32(self, v, out, stream=None):
        """y = S v in FP32 (float32 tensors; needs factor(precision=1))."""
        return self._op("smpm_apply_schur32", v, out, stream, dtype="float32")

    def apply_schur_class(self, v, out, stream=None):
        """y = S v by the element-class-shared path (float64 tensors)."""
        return self._op("smpm_apply_schur_class", v, out, stream)

    def apply_schur_class32(self, v, out, stream=None):
        """y = S v in FP32 by the element-class-shared path (needs factor(precision=1))."""
        return self._op("smpm_apply_schur_class32", v, out, stream, dtype="float32")

    def apply_precond(self, v, out, stream=None):
        return self._op("smpm_apply_precond", v, out, stream)

    def apply_schur_precond(self, v, out, stream=None):
        return self._op("smpm_apply_schur_precond", v, out, stream)

    def apply_deflation(self, v, out, stream=None):
        return self._op("smpm_apply_deflation", v, out, stream)

    def apply_deflation_noalloc(self, v, out, stream=None):
        """y = P v through the entry point that allocates nothing (scratch in a
        static device array shared by all calls on a device)."""
        return self._op("smpm_apply_deflation_noalloc", v, out, stream)

    def apply_deflation_q(self, v, out, stream=None):
        return self._op("smpm_apply_deflation_q", v, out, stream)

    def schur_rhs(self, b, out, stream=None):
        return self._op("smpm_schur_rhs", b, out, stream, n_in=self.r)

    def recover(self, b, x, out, stream=None):
        check(lib().smpm_recover(self.h, _dev(b, self.r, "b"), _dev(x, self.kp, "x"), _dev(out, self.r, "out"),
                                 _stream(stream)))
        return out

    def null_vectors(self, uL, uS, uC, stream=None):
        check(lib().smpm_null_vectors(self.h, _dev(uL, self.r, "uL", optional=True),
                                      _dev(uS, self.kp, "uS", optional=True), _dev(uC, self.d, "uC", optional=True),
                                      _stream(stream)))


def set_barrier_spin_limit(spins):
    """smpm_set_barrier_spin_limit: polls of every device-side barrier wait
    before it times out (spins <= 0 restores the default); a testing hook."""
    check(lib().smpm_set_barrier_spin_limit(int(spins)))


def factor_many(grids, stream=None, **opts):
    """schur_factor for many grids with the same options; the host factor
    steps run in parallel."""
    o = default_opts(**opts)
    hs = (ctypes.c_void_p * len(grids))(*[g.h for g in grids])
    check(lib().smpm_factor_many(hs, len(grids), ctypes.byref(o), _stream(stream)))
    for g in grids:
        g.opts = o
        g.factored = True


class Batch:
    """Many factored grids (and right-hand sides) solved in one persistent
    launch (smpm_batch_*).  f, g, u are packed problem-major: problem p's
    k-th right-hand side starts at offsets()[p] + k * r_p (g: with kp)."""

    def __init__(self, grids, nrhs, team_size=0, use_graph=True, precision=-1):
        self.grids = list(grids)
        self.nrhs = [int(k) for k in nrhs]
        hs = (ctypes.c_void_p * len(self.grids))(*[g.h for g in self.grids])
        ks = (ctypes.c_int * len(self.grids))(*self.nrhs)
        b = ctypes.c_void_p()
        check(lib().smpm_batch_create(hs, len(self.grids), ks, int(team_size), 1 if use_graph else 0,
                                      int(precision), ctypes.byref(b)))
        self.b = b
        info = self.info()
        self.f_len, self.g_len, self.ntasks = info["f_len"], info["g_len"], info["ntasks"]

    def info(self):
        fl, gl, nt = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        ts, nteams, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        check(lib().smpm_batch_info(self.b, ctypes.byref(fl), ctypes.byref(gl), ctypes.byref(nt), ctypes.byref(ts),
                                    ctypes.byref(nteams), ctypes.byref(ms)))
        return {"f_len": fl.value, "g_len": gl.value, "ntasks": nt.value, "team_size": ts.value,
                "nteams": nteams.value, "last_ms": ms.value}

    def offsets(self, kind="f"):
        """Start of each problem's block in the packed f/u ("f") or g ("g")."""
        out, o = [], 0
        for g, k in zip(self.grids, self.nrhs):
            out.append(o)
            o += k * (g.r if kind == "f" else g.kp)
        return out

    def solve(self, f, u, g=None, stream=None, allow_notconv=False):
        reps = (SmpmReport * self.ntasks)()
        st = lib().smpm_batch_solve(self.b, _dev(f, self.f_len, "f"), _dev(g, self.g_len, "g", optional=True),
                                    _dev(u, self.f_len, "u"), reps, _stream(stream))
        check(st, allow=(SMPM_ENOTCONV,) if allow_notconv else ())
        return [r.as_dict() for r in reps]

    def autotune(self, f, u, g=None, candidates=(8, 16, 19, 38, 76, 152), stream=None):
        cands = (ctypes.c_int * len(candidates))(*candidates)
        ms = (ctypes.c_double * len(candidates))()
        chosen = ctypes.c_int()
        check(lib().smpm_batch_autotune(self.b, _dev(f, self.f_len, "f"), _dev(g, self.g_len, "g", optional=True),
                                        _dev(u, self.f_len, "u"), _stream(stream), cands, len(candidates),
                                        ms, ctypes.byref(chosen)))
        return chosen.value, {c: ms[i] for i, c in enumerate(candidates)}

    def v_len(self):
        """Length of the packed slot vectors of apply_schur (sum of kp)."""
        return sum(g.kp for g in self.grids)

    def set_apply_kernel(self, kind):
        """1: warp per element from global memory (default); 0: bulk-copy ring."""
        check(lib().smpm_batch_set_apply_kernel(self.b, int(kind)))

    def apply_schur(self, v, y, stream=None):
        """y_p = S_p v_p for every problem (packed slot vectors, float64)."""
        n = self.v_len()
        check(lib().smpm_batch_apply_schur(self.b, _dev(v, n, "v"), _dev(y, n, "y"), _stream(stream)))
        return y

    def apply_schur32(self, v, y, stream=None):
        """As apply_schur with the FP32 factors (float32 vectors)."""
        n = self.v_len()
        check(lib().smpm_batch_apply_schur32(self.b, _dev(v, n, "v", "float32"), _dev(y, n, "y", "float32"),
                                             _stream(stream)))
        return y

    def task_times(self):
        """(team, start ms, end ms) of every right-hand side of the last solve."""
        team = np.empty(self.ntasks, dtype=np.int32)
        t0 = np.empty(self.ntasks)
        t1 = np.empty(self.ntasks)
        check(lib().smpm_batch_task_times(self.b, team.ctypes.data, t0.ctypes.data, t1.ctypes.data))
        return team, t0, t1

    def close(self):
        if getattr(self, "b", None):
            lib().smpm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
