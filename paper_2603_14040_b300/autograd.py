"""torch.autograd.Function around pyro_stokes_solve / pyro_stokes_adjoint.

Forward: (eta_n, eta_c, rho) -> (vx, vy, p) by the multigrid-preconditioned FGMRES solve.
Backward: one adjoint solve A lambda = dJ/dx (A is symmetric) and the fused strain-rate-product
kernel give dJ/deta_n, dJ/deta_c and dJ/drho. Parameterisations such as eta = exp(log_eta) or
eta_n = mean of the adjacent eta_c compose through torch as usual (dJ/dlog eta = eta dJ/deta).
"""
import itertools

import torch

from .pyro import Stokes, PyroError

_ids = itertools.count(1)


class StokesSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eta_n, eta_c, rho, solver, g, tol, adj_tol):
        shape = solver.shape
        out = [torch.zeros(shape, dtype=torch.float64, device=eta_n.device) for _ in range(3)]
        en, ec, rh = (t.detach().contiguous() for t in (eta_n, eta_c, rho))
        stats = solver.solve(en, ec, rh, g, tol, *out)
        sid = next(_ids)
        solver._last_solve_id = sid
        ctx.solver, ctx.g, ctx.tol, ctx.adj_tol, ctx.sid = solver, g, tol, adj_tol, sid
        ctx.stats = stats
        ctx.save_for_backward(en, ec, rh)
        return tuple(out)

    @staticmethod
    def backward(ctx, gvx, gvy, gp):
        en, ec, rh = ctx.saved_tensors
        solver = ctx.solver
        if getattr(solver, "_last_solve_id", None) != ctx.sid:
            # the handle has solved something else since: restore this state by solving again
            tmp = [torch.zeros(solver.shape, dtype=torch.float64, device=en.device) for _ in range(3)]
            solver.solve(en, ec, rh, ctx.g, ctx.tol, *tmp)
            solver._last_solve_id = ctx.sid
        zero = lambda: torch.zeros(solver.shape, dtype=torch.float64, device=en.device)
        gvx = gvx.contiguous() if gvx is not None else zero()
        gvy = gvy.contiguous() if gvy is not None else zero()
        gp = gp.contiguous() if gp is not None else zero()
        gn, gc, gr = zero(), zero(), zero()
        solver.adjoint(gvx, gvy, gp, ctx.adj_tol, gn, gc, gr)
        return gn, gc, gr, None, None, None, None


def stokes_solve(eta_n, eta_c, rho, solver, g=(0.0, 1.0), tol=1e-10, adj_tol=None):
    """Differentiable solve; returns (vx, vy, p)."""
    return StokesSolve.apply(eta_n, eta_c, rho, solver, tuple(g), float(tol),
                             float(adj_tol if adj_tol is not None else tol))


def surface_misfit(vx, vx_obs):
    """J = 1/2 sum_j (vx(1, j) - vx_obs(j))^2 over the vx unknowns of the top cell row."""
    nx = vx.shape[1] - 2
    d = vx[1, 1:nx] - vx_obs[1:nx]
    return 0.5 * torch.sum(d * d)


def node_from_cell(eta_c):
    """eta_n(i,j) = mean of the (up to four) cells adjacent to basic node (i,j) (a parameterisation
    in which only eta_c is free)."""
    ny, nx = eta_c.shape[0] - 2, eta_c.shape[1] - 2
    c = eta_c[1:ny + 1, 1:nx + 1]
    pad = torch.nn.functional.pad(c, (1, 1, 1, 1))
    ones = torch.nn.functional.pad(torch.ones_like(c), (1, 1, 1, 1))
    s = pad[:-1, :-1] + pad[:-1, 1:] + pad[1:, :-1] + pad[1:, 1:]
    w = ones[:-1, :-1] + ones[:-1, 1:] + ones[1:, :-1] + ones[1:, 1:]
    en = torch.zeros_like(eta_c)
    en[:ny + 1, :nx + 1] = s / w
    return en
