"""Plain FP64 CPU oracle for the deflated Schur-complement solve of the SMPM
Poisson-Neumann system (Joshi & Diamessis, arXiv 1601.03432).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library: it has its own GLL nodes, differentiation matrix,
operator assembly, factorisations and GMRES.

Every function follows the paper's definitions in the paper's order and cites
the passage it implements.  Library primitives (dense LU, sparse LU, SVD, matrix
products) serve as single steps; there is no blocking, fusion or reordering
beyond what the paper's definitions state.

Modules
-------
gll      GLL nodes, weights, differentiation matrix (Sec. 1.2).
smpm     Grid, element residual of Eq. (smpm_poisson), the split L = A + EB
         (Sec. 1.3), right-hand side f + tau g.
schur    S = I + B A^-1 E (Eq. schur_complement_system), null vectors u_L, u_S
         (Sec. 1.4), block-Jacobi M (Sec. 2, Fig. 2), deflation Z, C, P, Q
         (Eqs. projection1/projection2) and the regularised coarse solve.
gmres    Restarted GMRES with modified Gram-Schmidt and Givens rotations.
methods  Algorithms 1, 2, 3, the direct bordered solve of L u = f~ and the
         zero-mean normalisation.
adjoint  Reverse-mode derivative of u(f, g): the transposed bordered direct
         solve and Algorithm 3 on S^T (transposed blocks, C^T, swapped null
         vectors), with dl/df and dl/dg.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(closed forms, the Fig. 1 node list, the operator L entry by entry against a
hand derivation for n = 2 and a derivation from Lagrange polynomials in
physical coordinates for n <= 5 -- which pins the penalty and the Robin
identity weight under both readings --, polynomial exactness, spectral
convergence, operator identities, agreement of Algorithms 1-3 with the direct
solve, GMRES's minimal-residual definition checked by least squares on the
Krylov space; for the adjoint, brute-force transposition of the forward map,
the inner-product identity and central differences).  Planted mistakes in the
operator, the Schur and deflation objects, the algorithms, GMRES and the
adjoint are each caught by one of those pins.  No function is "parity unpinned".
"""
