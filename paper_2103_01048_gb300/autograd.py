"""torch.autograd.Function around pb_solve / pb_solvation_energy / pb_energy_grad.

Forward: the polar solvation energy (Eq. energy, kcal/mol) of point charges
`q` [na] at positions `x` [na, 3] inside a fixed surface mesh.  Backward:
dE/dq and dE/dx from one adjoint solve in the library (the surface is held
fixed).  Argument marshalling only; all arithmetic runs in libpbfmm.so.
"""
import numpy as np
import torch

from . import (PB_MIXED, pb_energy_grad, pb_result_destroy, pb_solvation_energy, pb_solve)


class SolvationEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, q, x, pbctx, mesh, eps_in, eps_out, kappa, tol, precision, max_iter):
        qa = q.detach().double().cpu().numpy()
        xa = x.detach().double().cpu().numpy().reshape(-1, 3)
        res, _ = pb_solve(pbctx, mesh, xa, qa, eps_in, eps_out, kappa, tol, max_iter, precision=precision)
        try:
            e = pb_solvation_energy(pbctx, res)
            gq, gx, _ = pb_energy_grad(pbctx, res, len(qa), tol=tol, max_iter=max_iter)
        finally:
            pb_result_destroy(res)
        ctx_.save_for_backward(torch.from_numpy(gq).to(q), torch.from_numpy(gx).to(x))
        return torch.tensor(e, dtype=torch.float64, device=q.device)

    @staticmethod
    def backward(ctx_, g):
        gq, gx = ctx_.saved_tensors
        return g * gq, g * gx, None, None, None, None, None, None, None, None


def solvation_energy(q, x, pbctx, mesh, eps_in=4.0, eps_out=80.0, kappa=0.125, tol=1e-8, precision=PB_MIXED,
                     max_iter=500):
    """Differentiable polar solvation energy (kcal/mol)."""
    return SolvationEnergy.apply(q, x, pbctx, mesh, eps_in, eps_out, kappa, tol, precision, max_iter)
