"""Writes the stored oracle references of the full-size parity tests:
sampled entries of the zero-mean solution of the oracle's Algorithm 3
(Sec. 2, Eq. deflated_schur; FP64, GMRES(50)) for

* the 32 x 32 element, n = 24 grid with the Fourier right-hand sides of
  seeds 1000 (to a relative 1e-12) and 1001 (to 1e-11: FP64 GMRES(50)
  stagnates near 1e-12 on this one and needs 652 steps to reach it),
* the 48 x 48 element, n = 16 grid with the Fourier right-hand side of
  seed 6 (the forward solve of the adjoint workload), to a relative 1e-11
  (FP64 GMRES stagnates near 3e-12 on this grid).

Each file holds the grid, the seed, the oracle's iteration count, the L2 norm
of the whole solution, and every `stride`-th entry (index, value).  Only the
oracle and the seeded input generators are called.  Setup takes several
minutes per grid (sparse LU of the bordered S^T for u_S).

    python tests/golden/make_fullsize_refs.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle.smpm import SMPMGrid  # noqa: E402
from oracle.schur import SchurSystem  # noqa: E402
from oracle import methods  # noqa: E402
from paper_1601_03432_gb300 import inputs  # noqa: E402

CASES = [
    ("config3_32x32_n24", (32, 32, 24), [(1000, 1e-12), (1001, 1e-11)]),
    ("config5_48x48_n16", (48, 48, 16), [(6, 1e-11)]),
]
STRIDE = 997


def main():
    for name, (mx, my, n), seeds in CASES:
        t0 = time.time()
        g = SMPMGrid(mx, my, n)
        s = SchurSystem(g)
        x, y = g.coords()
        print(name, "setup %.0f s" % (time.time() - t0), flush=True)
        for seed, tol in seeds:
            f, _ = inputs.fourier_rhs(x, y, seed=seed)
            u, info = methods.algorithm3(s, f, tol=tol, restart=50, maxit=2000)
            assert info["converged"], info
            path = os.path.join(HERE, "%s_fourier%d.txt" % (name, seed))
            with open(path, "w") as fh:
                fh.write("# oracle Algorithm 3 (FP64, GMRES(50), relative tol %.0e), zero-mean u\n" % tol)
                fh.write("# written by tests/golden/make_fullsize_refs.py\n")
                fh.write("mx %d my %d n %d seed %d iterations %d stride %d r %d tol %.0e\n"
                         % (mx, my, n, seed, info["iterations"], STRIDE, g.r, tol))
                fh.write("norm2 %.17e\n" % np.linalg.norm(u))
                for i in range(0, g.r, STRIDE):
                    fh.write("%d %.17e\n" % (i, u[i]))
            print(path, info["iterations"], "%.0f s" % (time.time() - t0), flush=True)


if __name__ == "__main__":
    main()
