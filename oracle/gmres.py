"""Restarted GMRES (the Krylov solver Algorithms 1-3 call; the paper names it
only as GMRES and states a relative tolerance of 1e-10, Sec. 3.2).

Reading of what the paper leaves open: restarted GMRES(m) from x0 = 0,
Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg matrix,
stop when the rotated residual estimate |g_{j+1}| <= tol * ||b||; the true
residual is recomputed at every restart.  Iterations are counted as Arnoldi
steps.  A "happy" breakdown is taken when h_{j+1,j} <= 1e-14 * ||A v_j||.
"""
import numpy as np


def gmres(apply_op, b, tol, restart=50, maxit=1000, x0=None):
    """Solve apply_op(x) = b.  Returns x and a dict with the iteration count,
    convergence flag, the residual-estimate history (relative to ||b||) and the
    final true relative residual."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    info = {"iterations": 0, "converged": False, "history": [], "breakdown": False}
    if bnorm == 0.0:
        info["converged"] = True
        info["true_relres"] = 0.0
        return x, info
    target = tol * bnorm
    r = b - apply_op(x) if x0 is not None else b.copy()
    total = 0
    while True:
        beta = np.linalg.norm(r)
        if beta <= target:
            info["converged"] = True
            break
        if total >= maxit:
            break
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        V[0] = r / beta
        j_done = 0
        stop = False
        for j in range(m):
            w = apply_op(V[j])
            wnorm0 = np.linalg.norm(w)
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            hsub = H[j + 1, j]
            for i in range(j):                     # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            hnorm = np.hypot(H[j, j], H[j + 1, j])
            breakdown = hsub <= 1e-14 * wnorm0
            cs[j] = H[j, j] / hnorm
            sn[j] = H[j + 1, j] / hnorm
            H[j, j] = hnorm
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            total += 1
            j_done = j + 1
            info["history"].append(abs(gvec[j + 1]) / bnorm)
            if abs(gvec[j + 1]) <= target:
                info["converged"] = True
                stop = True
            if breakdown:
                info["breakdown"] = True
                stop = True
            if stop or total >= maxit:
                break
            V[j + 1] = w / hsub
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):         # back substitution
            y[i] = (gvec[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        x = x + V[:j_done].T @ y
        r = b - apply_op(x)
        if stop or total >= maxit:
            if info["breakdown"] and np.linalg.norm(r) <= target:
                info["converged"] = True
            break
    info["iterations"] = total
    info["true_relres"] = float(np.linalg.norm(r) / bnorm)
    return x, info
