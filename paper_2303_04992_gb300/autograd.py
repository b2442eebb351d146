"""torch.autograd binding of the solve: the interface-solve velocity as a
differentiable function of the boundary data.  Forward is kfbim_solve, backward
kfbim_solve_adjoint (GMRES on the transposed matvec); both run in the CUDA
library, this module only moves tensors."""
import torch


class _SolveVelocity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, solver, fpts, fgrid):
        N3 = solver.N ** 3
        phi = torch.zeros(solver.n_primary, dtype=torch.float64, device=g.device)
        u = torch.zeros(3 * N3, dtype=torch.float64, device=g.device)
        p = torch.zeros(N3, dtype=torch.float64, device=g.device)
        solver.solve(g.detach().contiguous(), phi, fpts, fgrid, u, p)
        ctx.solver = solver
        return u

    @staticmethod
    def backward(ctx, ubar):
        solver = ctx.solver
        gbar = torch.zeros(solver.n_primary, dtype=torch.float64, device=ubar.device)
        solver.solve_adjoint(ubar.contiguous(), gbar)
        return gbar, None, None, None


def solve_velocity(solver, g, fpts=None, fgrid=None):
    """u (3 N^3 face-grid velocity, values at Omega nodes are u_h) of the
    interior Dirichlet problem with boundary data g (n_primary, float64 CUDA
    tensor); differentiable in g.  fpts, fgrid: optional forcing (constant)."""
    return _SolveVelocity.apply(g, solver, fpts, fgrid)
