"""torch.autograd bridge: f(rho) with its gradient from the library's adjoint (Sec. 5.1).

forward: nc_set_design (PDE filter, RAMP) -> nc_solve_state (damped Newton) -> nc_objective.
backward: nc_solve_adjoint (J^T lambda = df/ds) -> nc_sensitivities (chain rule through RAMP and the
filter transpose), scaled by the incoming gradient. The problem must not be used for another design
between forward and backward.
"""

import torch

from ._abi import NC_OBJ_MEAN_T_HEATED
from .problem import Problem


class NatConvObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, problem, objective=NC_OBJ_MEAN_T_HEATED):
        problem.set_design(rho)
        problem.solve_state()
        f = problem.objective(objective)
        ctx.problem = problem
        ctx.objective = objective
        return torch.tensor(f, dtype=torch.float64, device=rho.device if rho.is_cuda else problem.device)

    @staticmethod
    def backward(ctx, grad_out):
        pb = ctx.problem
        pb.solve_adjoint(ctx.objective)
        g = pb.sensitivities()
        return (grad_out.to(g.device) * g).to(grad_out.device if grad_out.is_cuda else g.device), None, None


def objective(rho: torch.Tensor, problem: Problem, objective: int = NC_OBJ_MEAN_T_HEATED) -> torch.Tensor:
    """The objective (default: mean temperature over the heated region; NC_OBJ_SUPG_COMPLIANCE: the
    thermal compliance of Eq. objdiscr) for design rho (E values in [0, 1]); differentiable."""
    return NatConvObjective.apply(rho, problem, objective)
