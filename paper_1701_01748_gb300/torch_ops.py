"""Phi as a torch.autograd.Function whose backward is the library's Phi^dagger.

Forward: y = Phi x = Theta G F Z x (Section 2), computed by ``ppd_op_forward``
on the tensor's CUDA stream.  Backward: for a real input x and the
conjugate-Wirtinger convention torch uses for complex outputs, the gradient
of a real loss with respect to x is Re(Phi^H g) = Phi^dagger g, computed by
``ppd_op_adjoint``.  Tensors stay on the device; PyTorch only owns memory
and streams.
"""
from __future__ import annotations

import torch

from . import ppd


class PhiFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, solver: "ppd.Solver"):
        real = torch.float32 if solver.cfg.precision == ppd.PPD_FP32_FP64NORMS else torch.float64
        if x.dtype != real or not x.is_cuda:
            raise TypeError(f"Phi expects a CUDA {real} tensor")
        x = x.contiguous()
        y = torch.empty((solver.M, 2), dtype=real, device=x.device)
        s = torch.cuda.current_stream(x.device).cuda_stream
        ppd.ppd_op_forward(solver.ctx, x.data_ptr(), y.data_ptr(), s)
        ctx.solver = solver
        return torch.view_as_complex(y)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        solver = ctx.solver
        gr = torch.view_as_real(g.contiguous()).contiguous()
        out = torch.empty((solver.L, solver.L1), dtype=gr.dtype, device=gr.device)
        s = torch.cuda.current_stream(gr.device).cuda_stream
        ppd.ppd_op_adjoint(solver.ctx, gr.data_ptr(), out.data_ptr(), s)
        return out, None


def phi(x: torch.Tensor, solver: "ppd.Solver") -> torch.Tensor:
    """y = Phi x (differentiable; backward = Phi^dagger)."""
    return PhiFunction.apply(x, solver)
