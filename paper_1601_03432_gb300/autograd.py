"""torch.autograd binding of the solve: u = solve(f, g) with a backward pass
that is the library's adjoint solve (schur_solve_adjoint: Algorithm 3 on the
transposed Schur system).  Marshalling only: both passes run in libsmpm.so.

The solve is linear in (f, g), so the backward pass needs no saved
activations, only the factored grid (built with FLAG_ADJOINT).
"""
import torch

from ._binding import FLAG_ADJOINT, SmpmError  # noqa: F401


def _rows(x, width, name):
    if x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError("%s must be a float64 CUDA tensor" % name)
    if x.dim() == 1:
        x = x.unsqueeze(0)
    if x.dim() != 2 or x.shape[1] != width:
        raise ValueError("%s must have shape (%d,) or (nrhs, %d)" % (name, width, width))
    return x.contiguous()


class SchurSolve(torch.autograd.Function):
    """forward: u = schur_solve(f, g); backward: (dl/df, dl/dg) = schur_solve_adjoint(dl/du)."""

    @staticmethod
    def forward(ctx, grid, f, g, tol):
        squeeze = f.dim() == 1
        f2 = _rows(f, grid.r, "f")
        g2 = _rows(g, grid.kp, "g") if g is not None else None
        if g2 is not None and g2.shape[0] != f2.shape[0]:
            raise ValueError("f and g hold different numbers of right-hand sides")
        u = torch.empty_like(f2)
        ctx.reports = grid.solve(f2, u, g=g2, tol=tol, nrhs=f2.shape[0])
        ctx.grid, ctx.tol, ctx.squeeze = grid, tol, squeeze
        return u[0] if squeeze else u

    @staticmethod
    def backward(ctx, gu):
        grid = ctx.grid
        gu2 = _rows(gu, grid.r, "dl/du")
        gf = torch.empty_like(gu2)
        gg = torch.empty(gu2.shape[0], grid.kp, dtype=torch.float64, device=gu2.device) \
            if ctx.needs_input_grad[2] else None
        grid.solve_adjoint(gu2, gf, gg, tol=ctx.tol, nrhs=gu2.shape[0])
        if ctx.squeeze:
            gf = gf[0]
            gg = gg[0] if gg is not None else None
        return None, gf, gg, None


def schur_solve(grid, f, g=None, tol=0.0):
    """Differentiable zero-mean solve of the SMPM Poisson-Neumann system.
    f: (r,) or (nrhs, r) float64 CUDA tensor; g: the matching Neumann data per
    padded slot or None; grid factored with flags=FLAG_ADJOINT for backward."""
    return SchurSolve.apply(grid, f, g, tol)
