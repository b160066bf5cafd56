"""Planted mistakes in the oracle's restarted GMRES: each plausible error,
planted by editing one line of the oracle's own source at run time, must
make one of the GMRES pins fail.  The pins come from the definition of
GMRES, not from the oracle's code: the solution of a dense system (with
restarts), the minimal residual over each Krylov space by least squares on an
orthonormal basis, the true residual of the returned iterate equal to that
minimum, and termination in at most 3 steps when A has 3 distinct
eigenvalues."""
import os

import numpy as np
import pytest

import oracle.gmres as og

SRC = open(os.path.join(os.path.dirname(og.__file__), "gmres.py")).read()


def mutated_gmres(old=None, new=None):
    """The oracle's gmres recompiled from its source, with the single
    occurrence of `old` replaced by `new` (unchanged when old is None)."""
    src = SRC
    if old is not None:
        assert SRC.count(old) == 1, old
        src = SRC.replace(old, new)
    ns = {}
    exec(compile(src, "gmres_mutated.py", "exec"), ns)
    return ns["gmres"]


def first_failing_gmres_pin(gmres):
    rng = np.random.default_rng(3)
    n = 30
    A = np.eye(n) * 2 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    # the solution, through several restart cycles
    x, info = gmres(lambda v: A @ v, b, 1e-12, restart=5, maxit=300)
    if not info["converged"] or np.linalg.norm(x - np.linalg.solve(A, b)) > 1e-9 * np.linalg.norm(x):
        return "dense solve"
    # minimal residual over K_j for j = 1..10
    _, info = gmres(lambda v: A @ v, b, 1e-14, restart=n, maxit=10)
    k = b / np.linalg.norm(b)
    K = []
    for j in range(10):
        K.append(k)
        k = A @ k
        k = k / np.linalg.norm(k)
    for j in range(1, 11):
        Q, _ = np.linalg.qr(np.array(K[:j]).T)
        c, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        rmin = np.linalg.norm(b - A @ (Q @ c)) / np.linalg.norm(b)
        if len(info["history"]) < j or abs(info["history"][j - 1] - rmin) > 1e-10 + 1e-8 * rmin:
            return "minimal residual"
    # after one cycle the returned iterate's true residual is the rotated estimate
    if abs(info["true_relres"] - info["history"][-1]) > 1e-10 + 1e-8 * info["history"][-1]:
        return "estimate = true residual"
    # three distinct eigenvalues: at most three steps
    X = rng.standard_normal((n, n)) + np.sqrt(n) * np.eye(n)
    A3 = X @ np.diag(np.repeat([1.0, 2.0, 3.5], 10)) @ np.linalg.inv(X)
    x, info = gmres(lambda v: A3 @ v, b, 1e-9, restart=n, maxit=n)
    if not info["converged"] or info["iterations"] > 3 or \
            np.linalg.norm(x - np.linalg.solve(A3, b)) > 1e-7 * np.linalg.norm(x):
        return "three eigenvalues"
    return None


MUTATIONS = [
    ("residual estimate sign", "gvec[j + 1] = -sn[j] * gvec[j]", "gvec[j + 1] = sn[j] * gvec[j]"),
    ("rotation sign", "H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]",
     "H[i + 1, j] = sn[i] * H[i, j] + cs[i] * H[i + 1, j]"),
    ("rotation cosine index", "cs[j] = H[j, j] / hnorm", "cs[j] = H[j + 1, j] / hnorm"),
    ("Gram-Schmidt index", "w = w - H[i, j] * V[i]", "w = w - H[i, j] * V[0]"),
    ("basis normalisation", "V[j + 1] = w / hsub", "V[j + 1] = w / wnorm0"),
    ("back substitution coupling", "y[i] = (gvec[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]",
     "y[i] = gvec[i] / H[i, i]"),
    ("update not accumulated over restarts", "x = x + V[:j_done].T @ y", "x = V[:j_done].T @ y"),
    ("stale residual at restart", "        r = b - apply_op(x)\n        if stop", "        r = b.copy()\n        if stop"),
]


def test_unmutated_gmres_pins_hold():
    assert first_failing_gmres_pin(og.gmres) is None
    assert first_failing_gmres_pin(mutated_gmres()) is None   # the recompiled source itself


@pytest.mark.parametrize("label,old,new", MUTATIONS, ids=[m[0].replace(" ", "_") for m in MUTATIONS])
def test_planted_gmres_mistake_is_caught(label, old, new):
    gm = mutated_gmres(old, new)
    try:
        failed = first_failing_gmres_pin(gm)
    except Exception as e:
        failed = "exception: %s" % e
    assert failed is not None, label
