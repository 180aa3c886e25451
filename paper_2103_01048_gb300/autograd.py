"""torch.autograd.Function around pb_solve / pb_solvation_energy / pb_energy_grad.

Forward: the polar solvation energy (Eq. energy, kcal/mol) of point charges
`q` [na] at positions `x` [na, 3] inside a fixed surface mesh, by one solve.
Backward: dE/dq and dE/dx from one adjoint solve in the library (the surface
is held fixed); the adjoint solve runs only when backward runs, on the
forward solve's result, which the graph keeps until then (release the
graph, by backward or by dropping the energy tensor, before destroying the
mesh or the context).  Argument marshalling only; all arithmetic runs in
libpbfmm.so.
"""
import weakref

import torch

from . import (PB_MIXED, pb_energy_grad, pb_result_destroy, pb_solvation_energy, pb_solve)


class _Result:
    """Owns a pb_result handle; frees it when the autograd graph lets go."""

    def __init__(self, handle, na):
        self.handle = handle
        self.na = na
        self._fin = weakref.finalize(self, pb_result_destroy, handle)

    def release(self):
        self._fin()


class SolvationEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, q, x, pbctx, mesh, eps_in, eps_out, kappa, tol, precision, max_iter):
        qa = q.detach().double().cpu().numpy()
        xa = x.detach().double().cpu().numpy().reshape(-1, 3)
        res, _ = pb_solve(pbctx, mesh, xa, qa, eps_in, eps_out, kappa, tol, max_iter, precision=precision)
        holder = _Result(res, len(qa))
        e = pb_solvation_energy(pbctx, res)
        if ctx_.needs_input_grad[0] or ctx_.needs_input_grad[1]:
            ctx_.res = holder
            ctx_.pbctx = pbctx
            ctx_.tol = tol
            ctx_.max_iter = max_iter
            ctx_.meta = (q.dtype, q.device, x.dtype, x.device, x.shape)
        else:
            holder.release()
        return torch.tensor(e, dtype=torch.float64, device=q.device)

    @staticmethod
    def backward(ctx_, g):
        holder = ctx_.res
        gq, gx, _ = pb_energy_grad(ctx_.pbctx, holder.handle, holder.na, tol=ctx_.tol, max_iter=ctx_.max_iter)
        holder.release()
        qdt, qdev, xdt, xdev, xshape = ctx_.meta
        gd = g.detach().to(torch.float64).cpu()
        dq = (gd * torch.from_numpy(gq)).to(dtype=qdt, device=qdev)
        dx = (gd * torch.from_numpy(gx)).reshape(xshape).to(dtype=xdt, device=xdev)
        return dq, dx, None, None, None, None, None, None, None, None


def solvation_energy(q, x, pbctx, mesh, eps_in=4.0, eps_out=80.0, kappa=0.125, tol=1e-8, precision=PB_MIXED,
                     max_iter=500):
    """Differentiable polar solvation energy (kcal/mol)."""
    return SolvationEnergy.apply(q, x, pbctx, mesh, eps_in, eps_out, kappa, tol, precision, max_iter)
