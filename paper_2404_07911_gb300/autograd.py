"""Differentiable unfitted operator: y = A(kappa) x as a torch.autograd.Function.

forward   y = A(kappa) x                      (uf_set_kappa_device + uf_vmult, FP64)
backward  dL/dx     = A(kappa)^T dL/dy        (uf_vmult_adjoint)
          dL/dkappa = [ (dL/dy)^T (dA/dkappa_e) x ]_e   (uf_kappa_gradient)

Nothing but x and kappa is kept for the backward pass: the backward kernels recompute the
quadrature-point values.  A is linear in kappa, so second derivatives in kappa vanish.
"""
import torch


class UnfittedPoissonFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, kappa, op):
        if x.dtype != torch.float64 or kappa.dtype != torch.float64:
            raise ValueError("the differentiable operator runs in FP64")
        op.set_kappa_device(kappa.detach())
        y = op.vmult(x.detach().contiguous())
        ctx.op = op
        ctx.save_for_backward(x, kappa)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, kappa = ctx.saved_tensors
        op = ctx.op
        op.set_kappa_device(kappa.detach())
        gy = gy.contiguous()
        gx = op.vmult_adjoint(gy) if ctx.needs_input_grad[0] else None
        gk = op.kappa_gradient(gy, x.detach().contiguous()) if ctx.needs_input_grad[1] else None
        return gx, gk, None


def unfitted_poisson(x, kappa, op):
    """y = A(kappa) x with gradients for x and kappa (op: an FP64 UnfittedOperator)."""
    return UnfittedPoissonFunction.apply(x, kappa, op)
