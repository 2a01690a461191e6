"""torch.autograd wrapper of the HB apply: forward = hb_apply, backward =
hb_apply_adjoint (the hand-written adjoint kernels).

For the C-linear map u = A s (A = h^2 K, Eq. m_v2v) PyTorch's complex
convention gives grad_s = A^H grad_u for a real loss, which is exactly what
hb_apply_adjoint computes.  Tensors are CUDA complex128 of shape (nrhs, N_v)
(one right-hand side per row = the column-major layout of the C ABI).
"""
import torch


class HBApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s, op, dense=False):
        s = s.contiguous()
        u = torch.empty_like(s)
        stream = torch.cuda.current_stream(s.device)
        (op.apply_dense if dense else op.apply)(s, u, s.shape[0], stream)
        ctx.op = op
        ctx.dense = dense
        return u

    @staticmethod
    def backward(ctx, grad_u):
        g = grad_u.contiguous()
        gs = torch.empty_like(g)
        stream = torch.cuda.current_stream(g.device)
        (ctx.op.apply_dense_adjoint if ctx.dense else ctx.op.apply_adjoint)(g, gs, g.shape[0], stream)
        return gs, None, None


def hb_apply(s, op, dense=False):
    """u = h^2 K s, differentiable in s."""
    return HBApply.apply(s, op, dense)
